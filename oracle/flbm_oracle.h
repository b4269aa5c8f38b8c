/*
 * flbm_oracle.h -- plain FP64 CPU oracle for the ghost-mode filtered
 * fluctuating lattice Boltzmann method (GMF-FLBM) on D3Q27.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this code; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no header, table or helper with the CUDA
 * path: every constant below is re-derived here from the paper's Tables I/II.
 *
 * Notation follows the paper (Sec. II): populations f_i, weights w_i,
 * velocities c_i (Table I), Hermite basis e_ki with normalisation b_k
 * (Table II), relaxation frequency omega = 1/tau, c_s^2 = 1/3.
 *
 * Layout: populations are SoA, f[i*N + n] with node n = x + nx*(y + ny*z),
 * absolute values (not deviations), FP64.
 */
#ifndef FLBM_ORACLE_H
#define FLBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_Q 27

/* collision schemes (Sec. III: BGK-FLBM, GMF-FLBM, Reg-FLBM) */
#define ORACLE_BGK 0
#define ORACLE_GMF 1
#define ORACLE_REG 2

typedef struct oracle_box oracle_box;

/* Lattice tables.  c: 27x3 ints (Table I, velocity order fixed by this
 * oracle), w: 27 weights, E: 27x27 row-major E[k*27+i] = e_ki evaluated from
 * the Table II polynomial expressions, b: the printed-relation normalisation
 * b_k = n_k! c_s^(2 n_k) / mu_k, nk/muk: order and multiplicity per mode.
 * Any pointer may be NULL. */
void oracle_tables(int *c, double *w, double *E, double *b, int *nk, int *muk);

/* Philox4x32-10 block function (Salmon et al., SC'11). */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The 23 standard normals r_4..r_26 of one node at one step (written to
 * r[4..26]; r[0..3] set to 0).  Counter = (node lo, step lo, block, step hi),
 * key = (seed lo, seed hi); block j word m feeds mode 4+4j+m; Box-Muller on
 * consecutive word pairs; uniform u = ((x >> 9) + 0.5) * 2^-23. */
void oracle_normals(uint64_t seed, uint64_t node, uint64_t step, double r[27]);
/* Same with a noise stream id in the high 24 bits of counter word 2 (block
 * j in the low 8 bits): independent streams under one seed; stream 0 is
 * oracle_normals. */
void oracle_normals_stream(uint64_t seed, uint32_t stream, uint64_t node, uint64_t step,
                           double r[27]);

/* Second-order equilibrium f^eq_i(rho, u). */
void oracle_feq2(double rho, const double u[3], double feq[27]);

/* Population-space noise term  w_i sum_k b_k^-1 e_ki phi_k r_k  for a node
 * of density rho, for the given scheme and tau, kT. */
void oracle_noise_term(int scheme, double tau, double kT, double rho,
                       const double r[27], double xi[27]);

/* Post-collision populations of one node (no streaming). */
void oracle_collide_node(int scheme, double tau, double kT, double rho_phi0,
                         int noise_rho0, uint64_t seed, uint64_t node,
                         uint64_t step, const double f[27], double fstar[27]);

/* Box life cycle.  create() initialises f_i = w_i rho0 at step 0. */
oracle_box *oracle_create(int nx, int ny, int nz, double tau, double kT,
                          double rho0, uint64_t seed, int scheme, int noise_rho0);
void oracle_destroy(oracle_box *b);
void oracle_set_populations(oracle_box *b, const double *f);
void oracle_get_populations(const oracle_box *b, double *f);
int64_t oracle_get_step(const oracle_box *b);
void oracle_set_step(oracle_box *b, int64_t step);
/* Noise stream id of the box (default 0); see oracle_normals_stream. */
void oracle_set_stream(oracle_box *b, uint32_t stream);
void oracle_step(oracle_box *b, int64_t n);

/* Advance n steps, recording the populations of node 0 before every step
 * into out[s*27 + i] (s = 0..n-1).  Used for the single-node AR(1) pins. */
void oracle_trajectory_node0(oracle_box *b, int64_t n, double *out);

/* Moments of the current (pre-collision) state: rho[N], j[3N] (x,y,z
 * planes), pi[6N] full second moment sum_i f_i c_ia c_ib in the order
 * xx, yy, zz, xy, xz, yz.  Any pointer may be NULL. */
void oracle_moments(const oracle_box *b, double *rho, double *j, double *pi);

/* Normalised-FFT structure factor of a real field m[N] (Sec. III):
 * dm(n) = N^-1/2 sum_x (m(x) - mean) exp(-2 pi i n.x / L), integer
 * wavevector n_a in [-L_a/2, L_a/2), shell s = round(|n|), n = 0 excluded.
 * S[s] = mean over the shell of |dm(n)|^2, count[s] = shell population,
 * s < nshell (larger shells dropped).  Naive separable DFT. */
void oracle_structure_factor(const double *m, int nx, int ny, int nz,
                             int nshell, double *S, int64_t *count);

/* OpenMP threads used by oracle_step / oracle_structure_factor (<=0: all). */
void oracle_set_threads(int n);
int oracle_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
