/*
 * flbm_oracle.c -- plain FP64 CPU oracle for GMF-FLBM on D3Q27.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product library.  It is written
 * to be read against the paper, not to be fast: every formula below is the
 * paper's, evaluated literally in population space, with no blocking, fusion
 * or sum factorisation.
 *
 *   Table I   : D3Q27 velocities and weights            -> VEL, weight()
 *   Table II  : full-Hermite basis e_ki, n_k, mu_k, b_k  -> hermite_e(), NK, MUK
 *   Eqs. rho/u: conserved moments                       -> collide()
 *   Eq. (2nd-order f^eq), Eq. moments2, Eq. f^neq       -> feq2(), collide()
 *   Eq. fluct_phi / fluct_phig: FDT amplitudes           -> noise_term()
 *   Eq. flbe2 : GMF-FLBM update (LHS = push streaming)   -> oracle_step()
 *   Eq. flbe  : BGK-FLBM update                          -> collide()
 *   Sec. III  : Reg-FLBM (full-order f^eq, mode-by-mode relaxation)
 *   Sec. III  : normalised-FFT spectra S_m(|k|)           -> oracle_structure_factor()
 *
 * Readings of points the paper leaves open (velocity order, RNG, which rho
 * enters phi_k, Reg-FLBM ghost relaxation) are stated where they are used.
 */
#include "flbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q ORACLE_Q
static const double CS2 = 1.0 / 3.0; /* c_s^2, Sec. II */

/* Table I.  The paper lists the velocity groups as sets; the order inside
 * each group is this oracle's reading: rest; +x,-x,+y,-y,+z,-z; the twelve
 * |c|^2=2 velocities as (xy),(xz),(yz) planes, each (+,+),(-,-),(+,-),(-,+);
 * the eight corners (+++),(---),(++-),(--+),(+-+),(-+-),(-++),(+--).
 * Opposite velocities are adjacent (i odd <-> i+1). */
static const int VEL[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},
    {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},
    {1, 1, 1},   {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
    {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1},
};

/* Table I weights by |c_i|^2. */
static double weight(int i)
{
    int s = VEL[i][0] * VEL[i][0] + VEL[i][1] * VEL[i][1] + VEL[i][2] * VEL[i][2];
    switch (s) {
    case 0: return 8.0 / 27.0;
    case 1: return 2.0 / 27.0;
    case 2: return 1.0 / 54.0;
    default: return 1.0 / 216.0;
    }
}

/* Table II: order n_k and multiplicity mu_k of mode k (listing order). */
static const int NK[Q] = {0, 1, 1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3,
                          4, 4, 4, 4, 4, 4, 5, 5, 5, 6};
static const int MUK[Q] = {1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 3, 3, 3, 3, 3, 3, 6,
                           6, 6, 6, 12, 12, 12, 30, 30, 30, 90};

/* Table II "Hermite symbols": the Cartesian indices of each mode's
 * polynomial, used for the Maxwell-Boltzmann Hermite coefficients
 * a_eq = rho u_a1 ... u_an of the Reg-FLBM equilibrium.  0=x, 1=y, 2=z. */
static const int HSYM[Q][6] = {
    {-1},                                   /* 0  H            */
    {0, -1}, {1, -1}, {2, -1},              /* 1-3 H_x,H_y,H_z  */
    {0, 0, -1}, {1, 1, -1}, {2, 2, -1},     /* 4-6 xx,yy,zz     */
    {0, 1, -1}, {0, 2, -1}, {1, 2, -1},     /* 7-9 xy,xz,yz     */
    {0, 0, 1, -1}, {0, 0, 2, -1},           /* 10,11 x^2y, x^2z */
    {1, 1, 0, -1}, {2, 2, 0, -1},           /* 12,13 y^2x, z^2x */
    {1, 1, 2, -1}, {2, 2, 1, -1},           /* 14,15 y^2z, z^2y */
    {0, 1, 2, -1},                          /* 16 xyz           */
    {0, 0, 1, 1, -1}, {0, 0, 2, 2, -1}, {1, 1, 2, 2, -1},   /* 17-19 */
    {0, 1, 2, 2, -1}, {0, 2, 1, 1, -1}, {1, 2, 0, 0, -1},   /* 20-22 */
    {0, 0, 1, 2, 2, -1}, {0, 0, 2, 1, 1, -1}, {1, 1, 0, 2, 2, -1}, /* 23-25 */
    {0, 0, 1, 1, 2, 2},                     /* 26 x^2y^2z^2     */
};

/* Table II, column e_ki, evaluated literally for velocity c = (cx,cy,cz). */
static double hermite_e(int k, const int *c)
{
    const double x = c[0], y = c[1], z = c[2];
    const double s = CS2;
    /* (alpha, beta[, gamma]) assignments of each group, listing order */
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    /* c_a c_b - c_s^2 delta_ab, diagonal */
    case 4: return x * x - s;
    case 5: return y * y - s;
    case 6: return z * z - s;
    /* off-diagonal */
    case 7: return x * y;
    case 8: return x * z;
    case 9: return y * z;
    /* c_a^2 c_b - c_s^2 c_b  for x^2y, x^2z, y^2x, z^2x, y^2z, z^2y */
    case 10: return x * x * y - s * y;
    case 11: return x * x * z - s * z;
    case 12: return y * y * x - s * x;
    case 13: return z * z * x - s * x;
    case 14: return y * y * z - s * z;
    case 15: return z * z * y - s * y;
    /* c_a c_b c_g */
    case 16: return x * y * z;
    /* c_a^2 c_b^2 - c_s^2 (c_a^2 + c_b^2) + c_s^4  for x^2y^2, x^2z^2, y^2z^2 */
    case 17: return x * x * y * y - s * (x * x + y * y) + s * s;
    case 18: return x * x * z * z - s * (x * x + z * z) + s * s;
    case 19: return y * y * z * z - s * (y * y + z * z) + s * s;
    /* c_a c_b c_g^2 - c_s^2 c_a c_b  for xyz^2, xzy^2, yzx^2 */
    case 20: return x * y * z * z - s * x * y;
    case 21: return x * z * y * y - s * x * z;
    case 22: return y * z * x * x - s * y * z;
    /* c_a^2 c_b c_g^2 - c_s^2 (c_a^2 c_b + c_b c_g^2) + c_s^4 c_b
     * for x^2yz^2 (a=x,b=y,g=z), x^2zy^2 (a=x,b=z,g=y), y^2xz^2 (a=y,b=x,g=z) */
    case 23: return x * x * y * z * z - s * (x * x * y + y * z * z) + s * s * y;
    case 24: return x * x * z * y * y - s * (x * x * z + z * y * y) + s * s * z;
    case 25: return y * y * x * z * z - s * (y * y * x + x * z * z) + s * s * x;
    /* c_a^2 c_b^2 c_g^2 - c_s^2 (pairs) + c_s^4 (squares) - c_s^6 */
    case 26:
        return x * x * y * y * z * z
             - s * (x * x * y * y + x * x * z * z + y * y * z * z)
             + s * s * (x * x + y * y + z * z) - s * s * s;
    default: return 0.0;
    }
}

static double factorial(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
}

/* b_k = n_k! c_s^(2 n_k) / mu_k  (Sec. II, relation after Eq. expneq) */
static double norm_b(int k)
{
    return factorial(NK[k]) * pow(CS2, NK[k]) / MUK[k];
}

/* Tables built once (the oracle is single-configuration, constants only). */
static double W[Q], E[Q][Q], B[Q];
static int tables_ready = 0;

static void build_tables(void)
{
    if (tables_ready) return;
    for (int i = 0; i < Q; ++i) W[i] = weight(i);
    for (int k = 0; k < Q; ++k) {
        B[k] = norm_b(k);
        for (int i = 0; i < Q; ++i) E[k][i] = hermite_e(k, VEL[i]);
    }
    tables_ready = 1;
}

void oracle_tables(int *c, double *w, double *e, double *b, int *nk, int *muk)
{
    build_tables();
    for (int i = 0; i < Q; ++i) {
        if (c) for (int a = 0; a < 3; ++a) c[3 * i + a] = VEL[i][a];
        if (w) w[i] = W[i];
        if (b) b[i] = B[i];
        if (nk) nk[i] = NK[i];
        if (muk) muk[i] = MUK[i];
        if (e) for (int j = 0; j < Q; ++j) e[i * Q + j] = E[i][j];
    }
}

/* ---------------------------------------------------------------------- */
/* Random numbers.  The paper asks only for standard normal r_k (Sec. II). */
/* Reading: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11 "Parallel      */
/* random numbers: as easy as 1, 2, 3") + Box-Muller (1958).                */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    /* round multipliers and Weyl key increments of Philox4x32 */
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * x0;
        uint64_t p1 = (uint64_t)M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* 23-bit uniform in (0,1), exactly representable in FP32 and FP64. */
static double uniform23(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

void oracle_normals_stream(uint64_t seed, uint32_t stream, uint64_t node, uint64_t step,
                           double r[27])
{
    const double two_pi = 2.0 * 3.14159265358979323846;
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int k = 0; k < 4; ++k) r[k] = 0.0;
    for (uint32_t j = 0; j < 6; ++j) {
        /* counter word 2: block j in the low 8 bits, noise stream above */
        uint32_t ctr[4] = {(uint32_t)node, (uint32_t)(step & 0xffffffffu), j | (stream << 8),
                           (uint32_t)(step >> 32)};
        uint32_t o[4];
        oracle_philox4x32_10(ctr, key, o);
        for (int p = 0; p < 2; ++p) {
            double u1 = uniform23(o[2 * p]);
            double u2 = uniform23(o[2 * p + 1]);
            double rad = sqrt(-2.0 * log(u1));
            int k = 4 + 4 * (int)j + 2 * p;
            r[k] = rad * cos(two_pi * u2);
            if (k + 1 < Q) r[k + 1] = rad * sin(two_pi * u2); /* mode 27 dropped */
        }
    }
}

void oracle_normals(uint64_t seed, uint64_t node, uint64_t step, double r[27])
{
    oracle_normals_stream(seed, 0u, node, step, r);
}

/* ---------------------------------------------------------------------- */
/* Collision.                                                               */

/* second-order equilibrium, Eq. after flbe2:
 * f^eq_i = w_i rho (1 + c_ia u_a / c_s^2 + (c_ia c_ib - c_s^2 d_ab) u_a u_b / (2 c_s^4)) */
void oracle_feq2(double rho, const double u[3], double feq[27])
{
    build_tables();
    for (int i = 0; i < Q; ++i) {
        double cu = 0.0, h2uu = 0.0;
        for (int a = 0; a < 3; ++a) {
            cu += VEL[i][a] * u[a];
            for (int b = 0; b < 3; ++b)
                h2uu += (VEL[i][a] * VEL[i][b] - CS2 * (a == b)) * u[a] * u[b];
        }
        feq[i] = W[i] * rho * (1.0 + cu / CS2 + h2uu / (2.0 * CS2 * CS2));
    }
}

/* phi_k of Eq. fluct_phi (k = 4..9, and all k for BGK-FLBM) and phi_k^g of
 * Eq. fluct_phig (k = 10..26 for GMF-FLBM and Reg-FLBM). */
static double phi_of(int scheme, int k, double omega, double kT, double rho)
{
    int ghost = k >= 10;
    if (ghost && scheme != ORACLE_BGK)
        return sqrt(rho * kT * B[k] / CS2);
    return sqrt(rho * kT * omega * (2.0 - omega) * B[k] / CS2);
}

void oracle_noise_term(int scheme, double tau, double kT, double rho,
                       const double r[27], double xi[27])
{
    build_tables();
    const double omega = 1.0 / tau;
    double phi[Q];
    for (int k = 0; k < Q; ++k) phi[k] = (k >= 4) ? phi_of(scheme, k, omega, kT, rho) : 0.0;
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int k = 4; k < Q; ++k) s += E[k][i] * phi[k] * r[k] / B[k];
        xi[i] = W[i] * s;
    }
}

static void collide(int scheme, double tau, double kT, double rho_phi0, int noise_rho0,
                    uint64_t seed, uint32_t stream, uint64_t node, uint64_t step,
                    const double *f, double *fstar)
{
    const double omega = 1.0 / tau;
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, u[3];
    for (int i = 0; i < Q; ++i) {                       /* Eqs. rho, u */
        rho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += f[i] * VEL[i][a];
    }
    for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;

    double r[Q], xi[Q];
    oracle_normals_stream(seed, stream, node, step, r);
    /* reading: phi_k uses the local density rho(x,t) (rho0 on request) */
    oracle_noise_term(scheme, tau, kT, noise_rho0 ? rho_phi0 : rho, r, xi);

    if (scheme == ORACLE_BGK) {
        /* Eq. flbe: f* = f^eq + (1-omega)(f - f^eq) + noise, 2nd-order f^eq */
        double feq[Q];
        oracle_feq2(rho, u, feq);
        for (int i = 0; i < Q; ++i)
            fstar[i] = feq[i] + (1.0 - omega) * (f[i] - feq[i]) + xi[i];
    } else if (scheme == ORACLE_GMF) {
        /* Eq. flbe2 with the filtered f^neq of Eqs. (f^neq, moments2) */
        double feq[Q], a2[3][3];
        oracle_feq2(rho, u, feq);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int i = 0; i < Q; ++i)
                    s += (f[i] - feq[i]) * (VEL[i][a] * VEL[i][b] - CS2 * (a == b));
                a2[a][b] = s;
            }
        for (int i = 0; i < Q; ++i) {
            double h2a = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    h2a += (VEL[i][a] * VEL[i][b] - CS2 * (a == b)) * a2[a][b];
            double fneq = W[i] * h2a / (2.0 * CS2 * CS2);
            fstar[i] = feq[i] + (1.0 - omega) * fneq + xi[i];
        }
    } else {
        /* Reg-FLBM (Sec. III): Eq. flbe2 with f^eq and f^neq expanded over the
         * full Hermite basis, Eqs. expeq / expneq / coeffneq, with
         * mu_k / (c_s^(2n_k) n_k!) = 1 / b_k.  Reading: the Maxwell-Boltzmann
         * Hermite coefficients a_eq = rho u_a1...u_an; mode-by-mode relaxation
         * (1-omega) for k = 4..9 and unit relaxation (no deterministic
         * memory) for the ghosts k = 10..26. */
        double aeq[Q], feq[Q], aneq[Q];
        for (int k = 0; k < Q; ++k) {
            double p = rho;
            for (int m = 0; m < 6 && HSYM[k][m] >= 0; ++m) p *= u[HSYM[k][m]];
            aeq[k] = p;
        }
        for (int i = 0; i < Q; ++i) {
            double s = 0.0;
            for (int k = 0; k < Q; ++k) s += E[k][i] * aeq[k] / B[k];
            feq[i] = W[i] * s;
        }
        for (int k = 0; k < Q; ++k) {
            double s = 0.0;
            for (int i = 0; i < Q; ++i) s += (f[i] - feq[i]) * E[k][i];
            aneq[k] = s;
        }
        for (int i = 0; i < Q; ++i) {
            double s = 0.0;
            for (int k = 4; k <= 9; ++k) s += (1.0 - omega) * E[k][i] * aneq[k] / B[k];
            fstar[i] = feq[i] + W[i] * s + xi[i];
        }
    }
}

void oracle_collide_node(int scheme, double tau, double kT, double rho_phi0,
                         int noise_rho0, uint64_t seed, uint64_t node,
                         uint64_t step, const double f[27], double fstar[27])
{
    build_tables();
    collide(scheme, tau, kT, rho_phi0, noise_rho0, seed, 0u, node, step, f, fstar);
}

/* ---------------------------------------------------------------------- */
/* Box: two arrays, push streaming f_i(x + c_i, t+1) = f*_i(x, t).          */

struct oracle_box {
    int nx, ny, nz;
    long long n;
    double tau, kT, rho0;
    uint64_t seed;
    int scheme, noise_rho0;
    uint32_t stream;
    int64_t step;
    double *f, *fn;
};

static int nthreads = 0;

void oracle_set_threads(int n) { nthreads = n; }

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    return 1;
#endif
}

oracle_box *oracle_create(int nx, int ny, int nz, double tau, double kT,
                          double rho0, uint64_t seed, int scheme, int noise_rho0)
{
    build_tables();
    if (nx < 1 || ny < 1 || nz < 1) return NULL;
    oracle_box *b = (oracle_box *)calloc(1, sizeof(oracle_box));
    if (!b) return NULL;
    b->nx = nx; b->ny = ny; b->nz = nz;
    b->n = (long long)nx * ny * nz;
    b->tau = tau; b->kT = kT; b->rho0 = rho0; b->seed = seed;
    b->scheme = scheme; b->noise_rho0 = noise_rho0;
    b->f = (double *)malloc(sizeof(double) * Q * b->n);
    b->fn = (double *)malloc(sizeof(double) * Q * b->n);
    if (!b->f || !b->fn) { oracle_destroy(b); return NULL; }
    for (int i = 0; i < Q; ++i)
        for (long long n = 0; n < b->n; ++n) b->f[i * b->n + n] = W[i] * rho0;
    return b;
}

void oracle_destroy(oracle_box *b)
{
    if (!b) return;
    free(b->f);
    free(b->fn);
    free(b);
}

void oracle_set_populations(oracle_box *b, const double *f)
{
    memcpy(b->f, f, sizeof(double) * Q * b->n);
}

void oracle_get_populations(const oracle_box *b, double *f)
{
    memcpy(f, b->f, sizeof(double) * Q * b->n);
}

int64_t oracle_get_step(const oracle_box *b) { return b->step; }
void oracle_set_stream(oracle_box *b, uint32_t stream) { b->stream = stream; }
void oracle_set_step(oracle_box *b, int64_t step) { b->step = step; }

static void one_step(oracle_box *b)
{
    const int nx = b->nx, ny = b->ny, nz = b->nz;
    const long long N = b->n;
#ifdef _OPENMP
    int nt = oracle_get_threads();
#pragma omp parallel for num_threads(nt) schedule(static)
#endif
    for (int z = 0; z < nz; ++z) {
        double f[Q], fs[Q];
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long long node = x + (long long)nx * (y + (long long)ny * z);
                for (int i = 0; i < Q; ++i) f[i] = b->f[i * N + node];
                collide(b->scheme, b->tau, b->kT, b->rho0, b->noise_rho0, b->seed, b->stream,
                        (uint64_t)node, (uint64_t)b->step, f, fs);
                for (int i = 0; i < Q; ++i) {
                    int xd = ((x + VEL[i][0]) % nx + nx) % nx;
                    int yd = ((y + VEL[i][1]) % ny + ny) % ny;
                    int zd = ((z + VEL[i][2]) % nz + nz) % nz;
                    long long dst = xd + (long long)nx * (yd + (long long)ny * zd);
                    b->fn[i * N + dst] = fs[i];
                }
            }
    }
    double *t = b->f; b->f = b->fn; b->fn = t;
    b->step += 1;
}

void oracle_step(oracle_box *b, int64_t n)
{
    for (int64_t s = 0; s < n; ++s) one_step(b);
}

void oracle_trajectory_node0(oracle_box *b, int64_t n, double *out)
{
    for (int64_t s = 0; s < n; ++s) {
        for (int i = 0; i < Q; ++i) out[s * Q + i] = b->f[i * b->n];
        one_step(b);
    }
}

void oracle_moments(const oracle_box *b, double *rho, double *j, double *pi)
{
    static const int PA[6] = {0, 1, 2, 0, 0, 1}, PB[6] = {0, 1, 2, 1, 2, 2};
    const long long N = b->n;
    for (long long n = 0; n < N; ++n) {
        double r = 0.0, jj[3] = {0, 0, 0}, p[6] = {0, 0, 0, 0, 0, 0};
        for (int i = 0; i < Q; ++i) {
            double f = b->f[i * N + n];
            r += f;
            for (int a = 0; a < 3; ++a) jj[a] += f * VEL[i][a];
            for (int q = 0; q < 6; ++q) p[q] += f * VEL[i][PA[q]] * VEL[i][PB[q]];
        }
        if (rho) rho[n] = r;
        if (j) for (int a = 0; a < 3; ++a) j[a * N + n] = jj[a];
        if (pi) for (int q = 0; q < 6; ++q) pi[q * N + n] = p[q];
    }
}

/* ---------------------------------------------------------------------- */
/* Structure factor: naive separable DFT, FP64.                            */

/* in-place 1D DFT of `len` complex values spaced by `stride` */
static void dft_line(double *re, double *im, long long base, long long stride, int len,
                     const double *cs, const double *sn, double *tr, double *ti)
{
    for (int k = 0; k < len; ++k) {
        double sr = 0.0, si = 0.0;
        for (int x = 0; x < len; ++x) {
            int ph = (int)(((long long)k * x) % len);
            double vr = re[base + x * stride], vi = im[base + x * stride];
            /* multiply by exp(-2 pi i k x / len) */
            sr += vr * cs[ph] + vi * sn[ph];
            si += vi * cs[ph] - vr * sn[ph];
        }
        tr[k] = sr; ti[k] = si;
    }
    for (int k = 0; k < len; ++k) { re[base + k * stride] = tr[k]; im[base + k * stride] = ti[k]; }
}

static void dft_axis(double *re, double *im, int nx, int ny, int nz, int axis)
{
    const double two_pi = 2.0 * 3.14159265358979323846;
    int len = axis == 0 ? nx : axis == 1 ? ny : nz;
    long long stride = axis == 0 ? 1 : axis == 1 ? nx : (long long)nx * ny;
    double *cs = (double *)malloc(sizeof(double) * len);
    double *sn = (double *)malloc(sizeof(double) * len);
    for (int p = 0; p < len; ++p) { cs[p] = cos(two_pi * p / len); sn[p] = sin(two_pi * p / len); }
    long long nlines = (long long)nx * ny * nz / len;
#ifdef _OPENMP
    int nt = oracle_get_threads();
#pragma omp parallel num_threads(nt)
#endif
    {
        double *tr = (double *)malloc(sizeof(double) * len);
        double *ti = (double *)malloc(sizeof(double) * len);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (long long l = 0; l < nlines; ++l) {
            long long base;
            if (axis == 0) base = l * nx;
            else if (axis == 1) base = (l % nx) + (l / nx) * (long long)nx * ny;
            else base = l;
            dft_line(re, im, base, stride, len, cs, sn, tr, ti);
        }
        free(tr); free(ti);
    }
    free(cs); free(sn);
}

static int wave_index(int k, int len) { return (2 * k < len) ? k : k - len; }

void oracle_structure_factor(const double *m, int nx, int ny, int nz,
                             int nshell, double *S, int64_t *count)
{
    const long long N = (long long)nx * ny * nz;
    double *re = (double *)malloc(sizeof(double) * N);
    double *im = (double *)calloc(N, sizeof(double));
    double mean = 0.0;
    for (long long n = 0; n < N; ++n) mean += m[n];
    mean /= (double)N;
    for (long long n = 0; n < N; ++n) re[n] = m[n] - mean;
    dft_axis(re, im, nx, ny, nz, 0);
    dft_axis(re, im, nx, ny, nz, 1);
    dft_axis(re, im, nx, ny, nz, 2);
    for (int s = 0; s < nshell; ++s) { S[s] = 0.0; count[s] = 0; }
    for (int kz = 0; kz < nz; ++kz)
        for (int ky = 0; ky < ny; ++ky)
            for (int kx = 0; kx < nx; ++kx) {
                long long a = wave_index(kx, nx), bb = wave_index(ky, ny), c = wave_index(kz, nz);
                long long n2 = a * a + bb * bb + c * c;
                if (n2 == 0) continue;
                int s = (int)lround(sqrt((double)n2));
                if (s >= nshell) continue;
                long long idx = kx + (long long)nx * (ky + (long long)ny * kz);
                S[s] += (re[idx] * re[idx] + im[idx] * im[idx]) / (double)N;
                count[s] += 1;
            }
    for (int s = 0; s < nshell; ++s)
        if (count[s] > 0) S[s] /= (double)count[s];
    free(re); free(im);
}
