/*
 * flbm.h -- C ABI of the GB300 (sm_103a) ghost-mode filtered fluctuating
 * lattice Boltzmann library (libflbm.so).
 *
 * The library advances a periodic nx*ny*nz D3Q27 box with the fluctuating
 * lattice Boltzmann update of Lauricella, Montessori, Tiribocchi, Succi,
 * "Ghost-Mode Filtered Fluctuating Lattice Boltzmann Method" (arXiv
 * 2601.03806):
 *   - GMF-FLBM, Eq. flbe2 (Sec. II): second-order f^eq, filtered f^neq
 *     (Eq. moments2), noise amplitudes phi_k (Eq. fluct_phi, k=4..9) and
 *     phi_k^g (Eq. fluct_phig, k=10..26);
 *   - BGK-FLBM, Eq. flbe (Sec. II): single relaxation of all modes;
 *   - Reg-FLBM (Sec. III): full-order Hermite f^eq, unit ghost relaxation.
 *
 * Conventions shared by every call
 *   - Every call returns an int status (flbm_status); no exception or
 *     longjmp crosses the ABI.  On failure the context's error string
 *     (flbm_last_error) says why.
 *   - Node index n = x + nx*(y + ny*z), x fastest.  Population arrays are
 *     SoA: f[i*N + n], N = nx*ny*nz, with the velocity order
 *        i = 0      (0,0,0)
 *        i = 1..6   +x -x +y -y +z -z
 *        i = 7..18  (+,+,0) (-,-,0) (+,-,0) (-,+,0)   xy plane
 *                   (+,0,+) (-,0,-) (+,0,-) (-,0,+)   xz plane
 *                   (0,+,+) (0,-,-) (0,+,-) (0,-,+)   yz plane
 *        i = 19..26 (+++) (---) (++-) (--+) (+-+) (-+-) (-++) (+--)
 *     (Table I groups; the order inside a group is this library's choice).
 *   - Host arrays are owned by the caller; the library never keeps a host
 *     pointer past the call.  Device memory is owned by the library unless
 *     flbm_create_ex is given dev_buf, which then must outlive the context.
 *   - Calls that return host data are synchronous on the context's stream.
 *     flbm_step returns after the launched steps completed (it reads the
 *     instability flag back).
 *   - Noise: Philox4x32-10 (Salmon et al., SC'11), key = (seed lo, seed hi),
 *     counter = (node, step lo, j | noise_stream << 8, step hi) for blocks
 *     j = 0..5; word m of block j
 *     feeds mode k = 4 + 4j + m (mode 27 unused); Box-Muller on consecutive
 *     word pairs with u = ((w >> 9) + 0.5) 2^-23.  The result therefore does
 *     not depend on launch shape, and a checkpoint (populations + step +
 *     seed) resumes bit-exactly.
 */
#ifndef FLBM_H
#define FLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FLBM_ABI_VERSION 1

typedef struct flbm_ctx flbm_ctx; /* opaque, owned by the library */

/* Collision scheme (Sec. III compares the first three).  FLBM_LEARNED is
 * this library's: GMF-FLBM plus a trained network's correction towards
 * Reg-FLBM (see "Learned collision" below); FP32 storage, kT > 0, and the
 * network set with flbm_set_mlp before the first step. */
enum flbm_scheme { FLBM_BGK = 0, FLBM_GMF = 1, FLBM_REG = 2, FLBM_LEARNED = 3 };

/* What a box keeps between steps (flbm_params.state_form).
 * POPULATIONS: the 27 populations, in place with the AA pattern (216 B of
 *   traffic per node and step in FP32).
 * MOMENTS: the paper's thread-safe formulation (end of Sec. II): per node
 *   the ten deterministic numbers of its last collision, rho - rho0, j and
 *   the relaxed second-order amplitudes, in two library-owned arrays of
 *   10 N floats; each step rebuilds the populations a node pulls from its
 *   neighbours' numbers and their regenerated noise (80 B of state traffic
 *   per node and step).  FP32, GMF or Reg only (BGK's ghost modes keep a
 *   memory of their own).  The results are those of the population form, bit
 *   for bit.  The population buffer stays: the first step after the
 *   populations were written collides from it, and any call that reads
 *   populations rebuilds them into it first. */
enum flbm_state_form { FLBM_STATE_POPULATIONS = 0, FLBM_STATE_MOMENTS = 1 };

/* Storage precision of the populations.
 * FLBM_FP64: deviations g_i = f_i - w_i rho0 in double, FP64 arithmetic.
 * FLBM_FP32: deviations in float, FP32 arithmetic (FP64 only for the global
 *            reductions and the S(k) accumulators).
 * FLBM_FP16: deviations in half (IEEE binary16, round to nearest), FP32
 *            arithmetic, FP64 reductions: 108 B of HBM traffic per lattice
 *            update instead of 216 B.  Raw-state calls use 16-bit halves. */
enum flbm_precision { FLBM_FP64 = 0, FLBM_FP32 = 1, FLBM_FP16 = 2 };

enum flbm_status {
    FLBM_OK = 0,
    FLBM_E_INVALID = -1,     /* bad argument (sizes, tau <= 0.5, kT < 0, ...) */
    FLBM_E_NOMEM = -2,       /* device or host allocation failed / buffer too small */
    FLBM_E_CUDA = -3,        /* a CUDA runtime / cuFFT call failed */
    FLBM_E_UNSTABLE = -4,    /* a step met rho <= 0 or a non-finite value */
    FLBM_E_TIMEOUT = -5,     /* reserved: bounded device wait ran out */
    FLBM_E_UNSUPPORTED = -6  /* valid request the library does not implement */
};

/* Observables of the equilibration ratio and of S(k) (Sec. III): the local
 * density, sum_a rho u_a, sum_a Pi_aa, sum_{a<b} Pi_ab, and the momentum
 * components. Pi_ab = sum_i f_i c_ia c_ib (full second moment). */
enum flbm_observable {
    FLBM_OBS_RHO = 0,
    FLBM_OBS_JSUM = 1,
    FLBM_OBS_PI_DIAG = 2,
    FLBM_OBS_PI_OFFDIAG = 3,
    FLBM_OBS_JX = 4,
    FLBM_OBS_JY = 5,
    FLBM_OBS_JZ = 6
};

typedef struct flbm_params {
    int32_t nx, ny, nz;    /* box, each >= 1; N * 27 < 2^40 */
    int32_t scheme;        /* flbm_scheme */
    int32_t precision;     /* flbm_precision */
    int32_t noise_rho0;    /* 0: phi_k uses the local rho(x,t); 1: uses rho0 */
    int32_t stats_every;   /* fused FP64 reductions every k-th step (0: off) */
    int32_t noise_stream;  /* noise stream id s, 0 <= s < 2^24: the Philox
                              counter word 2 is block | s << 8, so boxes under
                              one seed with distinct streams draw independent
                              noise (0: the default stream) */
    int32_t state_form;    /* flbm_state_form (0: populations) */
    double tau;            /* relaxation time, > 0.5 (omega = 1/tau) */
    double kT;             /* thermal energy k_B T >= 0 (lattice units) */
    double rho0;           /* reference density > 0; initial state f_i = w_i rho0 */
    uint64_t seed;         /* Philox key */
} flbm_params;

/* Statistics of the fused reductions (row a9).  Sums run over all nodes of
 * the pre-collision state f(x,t) of the reduced steps. */
typedef struct flbm_stats_t {
    int64_t step;          /* t of the most recent reduced step */
    int64_t n_samples;     /* reduced steps accumulated since flbm_stats_reset */
    double mass;           /* sum_x rho at that step */
    double mom[3];         /* sum_x rho u_a */
    double u2[3];          /* mean_x u_a^2 at that step */
    double u2_avg[3];      /* time average of u2 since reset */
    double m_mean[4];      /* time-space mean of (rho - rho0, sum j, sum_a Pi_aa - rho0,
                              sum_{a<b} Pi_ab) */
    double m_var[4];       /* their time-space variance */
    double er[4];          /* equilibration ratios m_var / theory, theory =
                              (3, 3, 5, 1) rho0 kT (lattice ideal-gas invariant
                              measure); 0 when kT = 0 */
} flbm_stats_t;

/* Fill p with defaults for a box: FP32 storage, local-rho noise, stats every
 * step.  Returns FLBM_E_INVALID on a NULL p. */
int flbm_params_init(flbm_params *p, int nx, int ny, int nz, double tau, double kT,
                     double rho0, uint64_t seed, int scheme);

/* Device bytes of the population state (AA-pattern in place): 27 slabs of
 * ns elements of the storage type, ns = flbm_state_bytes(p) / (27 x element
 * size) >= N; population slot i of node n is element i ns + n.  ns is N
 * rounded up to 64 elements plus a pad that keeps the 27 slabs from starting
 * at addresses equal in their low bits: 1 MiB for slabs of 32 MiB and more,
 * else none; FLBM_SLAB_PAD in the environment (bytes, a multiple of 128)
 * sets it at any size.  0 on invalid parameters.
 * A moment-state context (state_form = FLBM_STATE_MOMENTS) also allocates
 * 2 x 10 N floats of its own, which dev_buf does not cover. */
size_t flbm_state_bytes(const flbm_params *p);

/* Create a context with flbm_params_init defaults: FP32 deviations, AA in
 * place, library-owned memory and stream; state f_i = w_i rho0 at step 0.
 * The arguments are the run parameters of the paper's equilibrium-
 * fluctuation tests (Sec. III): a periodic nx x ny x nz box, the relaxation
 * time tau of the BGK collision (Sec. II: omega = 1/tau, shear viscosity
 * c_s^2 (tau - 1/2), tau > 1/2), the thermal energy kT of the fluctuation-
 * dissipation amplitudes (Eqs. fluct_phi, fluct_phig), the reference density
 * rho0, the key of the noise generator, and the scheme compared in Sec. III
 * (BGK-, GMF- or Reg-FLBM).  out receives the context (NULL on failure);
 * FLBM_E_INVALID on out-of-range parameters, FLBM_E_NOMEM / FLBM_E_CUDA when
 * the device allocation or set-up fails. */
int flbm_create(int nx, int ny, int nz, double tau, double kT, double rho0,
                uint64_t seed, int scheme, flbm_ctx **out);

/* Create from explicit parameters (the Sec. III run parameters of
 * flbm_create, plus storage precision, noise density reading, reduction
 * cadence, noise stream and state form; see flbm_params).  dev_buf: NULL, or
 * a device buffer, 256-byte aligned, that the caller (e.g. PyTorch) owns and
 * keeps alive: of at least flbm_state_bytes(p) bytes (padded slabs, as
 * described there), or of at least 27 N elements (unpadded slabs, ns = N;
 * FLBM_E_NOMEM below that); cuda_stream: NULL for
 * a library-owned stream, else a cudaStream_t on the current device that all
 * work of this context is ordered on.  FLBM_E_INVALID if dev_buf is not
 * device (or managed) memory or a parameter is out of range. */
int flbm_create_ex(const flbm_params *p, void *dev_buf, size_t dev_bytes,
                   void *cuda_stream, flbm_ctx **out);

/* Advance n >= 0 steps (Eq. flbe2 / flbe per the scheme; one fused
 * stream-and-collide kernel per step, reductions on the steps selected by
 * stats_every; in the moment-state form the first step after the
 * populations were written collides from them, later ones from the ten
 * numbers per node).  Returns FLBM_E_UNSTABLE if any step met rho <= 0 or a
 * non-finite density; the step counter is then the t of the first such
 * step and the populations hold that step's output (restore a checkpoint). */
int flbm_step(flbm_ctx *c, int64_t n);

/* Moments of the pre-collision state f(x, t) at the current step t (Eqs.
 * rho, u): rho[N], j[3N] (planes jx, jy, jz), pi[6N] (planes xx, yy, zz, xy,
 * xz, yz of Pi_ab = sum_i f_i c_ia c_ib).  Any pointer may be NULL. */
int flbm_moments(flbm_ctx *c, double *rho, double *j, double *pi);

/* Read the fused-reduction statistics (see flbm_stats_t). */
int flbm_stats(flbm_ctx *c, flbm_stats_t *out);

/* Restart the time averages (e.g. after a warm-up). */
int flbm_stats_reset(flbm_ctx *c);

/* Normalised-FFT spectrum of one observable of the current state (Sec. III):
 * dm(n) = N^-1/2 sum_x (m(x) - mean) exp(-2 pi i n.x / L) with integer
 * n_a in [-L_a/2, L_a/2); shell s = round(|n|), n = 0 excluded.  S[s] =
 * shell mean of |dm(n)|^2, count[s] = number of wavevectors, s < nshell
 * (larger shells dropped).  cuFFT R2C (FP32 storage) or D2Z (FP64), FP64
 * shell accumulation. */
int flbm_structure_factor(flbm_ctx *c, int observable, int nshell, double *S,
                          int64_t *count);

/* Spectral equilibration ratio of one observable of the current state (Sec.
 * III): ER_m(|k|) = S_m(|k|) / S_m^th with S_m as flbm_structure_factor
 * returns it and S_m^th the flat value of the lattice invariant measure per
 * node, (3, 3, 5, 1) rho0 kT for rho, sum_a j_a, sum_a Pi_aa, sum_{a<b}
 * Pi_ab and rho0 kT for each momentum component.  er[s] and count[s] for
 * shells s < nshell (er[s] = 0 for an empty shell).  FLBM_E_INVALID when
 * kT = 0 (no fluctuations to compare) and for the arguments
 * flbm_structure_factor rejects. */
int flbm_spectral_er(flbm_ctx *c, int observable, int nshell, double *er, int64_t *count);

/* Absolute populations f_i(x, t) of the current step, FP64, SoA f[i*N+n]. */
int flbm_get_populations(flbm_ctx *c, double *f);
int flbm_set_populations(flbm_ctx *c, const double *f);

/* Replace the state by a sample of the lattice ideal-gas invariant measure
 * of the fluctuating dynamics: independent Gaussian deviations
 * g_i(x) = sqrt(rho0 kT w_i / c_s^2) xi_i(x), xi ~ N(0,1), the stationary
 * population statistics that make every Hermite mode k carry its
 * equilibrium variance rho0 kT b_k / c_s^2 (the fluctuation-dissipation
 * balance behind Eqs. fluct_phi / fluct_phig).  Starting there skips the
 * thermalisation transient.  xi comes from Philox4x32-10 with key = seed and
 * counter (node, 0, block 6 + j, 0), j = 0..6, disjoint from the step noise
 * (blocks 0..5); Box-Muller on word pairs as for the noise; population i
 * takes normal i of the node.  The step counter is kept; storage is left in
 * the natural form. */
int flbm_init_thermal(flbm_ctx *c, uint64_t seed);

/* Absolute populations f_i(x, t) at `count` listed nodes (node indices n in
 * [0, N)), written as f[k*27 + i] for the k-th listed node: a probe for
 * large boxes where a full readback is impractical.  FLBM_E_INVALID if a
 * node index is out of range. */
int flbm_probe(flbm_ctx *c, const int64_t *nodes, int64_t count, double *f);

/* Raw state: deviations g_i = f_i - w_i rho0 in the storage type (double for
 * FLBM_FP64, float for FLBM_FP32, IEEE half for FLBM_FP16), SoA natural
 * layout, 27 N elements on the host (the device slabs' pads, see
 * flbm_state_bytes, are left out).
 * Checkpoint = get_state + flbm_get_step; restore = set_state + set_step. */
int flbm_get_state(flbm_ctx *c, void *host);
int flbm_set_state(flbm_ctx *c, const void *host);

/* Device timing of the fused step kernel.  While enabled, each step-kernel
 * launch is bracketed by two CUDA events recorded on the context stream (the
 * stream the kernel runs on).  flbm_timing_read waits for the recorded
 * events, returns the summed kernel time in milliseconds and the number of
 * timed launches since the last read/enable, and clears both. */
int flbm_timing_enable(flbm_ctx *c, int enable);
int flbm_timing_read(flbm_ctx *c, double *kernel_ms, int64_t *launches);

int64_t flbm_get_step(const flbm_ctx *c);       /* -1 on NULL */
int flbm_set_step(flbm_ctx *c, int64_t step);   /* step >= 0 */

/* Parameters the context was created with (copy). */
int flbm_get_params(const flbm_ctx *c, flbm_params *out);

/* Error text of the last failing call on c (context-owned, valid until the
 * next call on c); c == NULL gives the thread's last create-time error. */
const char *flbm_last_error(const flbm_ctx *c);

/* One fused step (the kernels of flbm_step) on caller-owned device memory,
 * with no device allocation: for callers that cannot let a library allocate
 * GPU memory, e.g. applications whose own allocator owns every byte of the
 * device, or a host program that embeds the solver under a fixed memory
 * budget.  The paper has no counterpart; this is a deployment interface.
 *
 *   p          box, scheme, tau, kT, rho0, seed, noise_rho0, noise_stream,
 *              checked as flbm_create checks them (FLBM_E_INVALID); precision
 *              must be FLBM_FP32, state_form FLBM_STATE_POPULATIONS and the
 *              scheme BGK, GMF or Reg (FLBM_E_UNSUPPORTED otherwise);
 *              stats_every ignored.  The launch shape is flbm_create's for
 *              the same box and environment (FLBM_ROWS, FLBM_CTAS_PER_SM), so
 *              populations and sums equal those of flbm_step + flbm_stats.
 *   dev_state  27 N floats of deviations g_i = f_i - w_i rho0, SoA planes,
 *              256-byte aligned, updated in place (AA pattern).
 *   step       time index t of this collision (the noise counter).
 *   parity     storage form of dev_state on entry: 0 natural (slot i of node
 *              x holds f_i(x)), 1 AA-shifted; the call leaves the other form.
 *   dev_sums   13 doubles of device memory receiving the global sums over the
 *              pre-collision state at t: drho, jx, jy, jz, ux^2, uy^2, uz^2,
 *              m3, m4, drho^2, (sum_a j_a)^2, m3^2, m4^2 with m3 = sum_a Pi_aa
 *              - rho0, m4 = sum_{a<b} Pi_ab.
 *   cuda_stream stream the work is ordered on (NULL: the legacy stream); the
 *              call returns after the step completed.
 * Scratch (per-CTA partial sums and flags) lives in one static device array
 * of 208 KiB that every GPU loading the library keeps until process exit;
 * a launch needing more than its 2048 CTA slots is rejected with
 * FLBM_E_INVALID.  The first call on a device resolves that array's address
 * (cudaGetSymbolAddress) with the device current and keeps it; make it
 * before any stream capture, and do not use the library on a device across
 * a cudaDeviceReset.  Every call reuses the same array, so calls that overlap on the
 * GPU (other streams, other threads) race and must be serialised by the
 * caller.  Errors: FLBM_E_INVALID, FLBM_E_UNSUPPORTED, FLBM_E_CUDA,
 * FLBM_E_UNSTABLE, FLBM_E_TIMEOUT; text via flbm_last_error(NULL). */
int flbm_step_noalloc(const flbm_params *p, void *dev_state, int64_t step, int parity,
                      double *dev_sums, void *cuda_stream);

/* Release everything the context owns (not a caller dev_buf/stream).  A
 * replica context of an ensemble is left alone (the ensemble owns it). */
void flbm_destroy(flbm_ctx *c);

/* ------------------------------------------------------------------------
 * Batched ensemble: many independent periodic boxes (replicas) of uneven
 * sizes, taus and noise streams advanced together by one persistent kernel
 * per step, for the ensemble averages that equilibrium fluctuation
 * statistics need (Sec. III measures <u^2> and S(k) as averages).  The
 * paper runs one box at a time; the ensemble is this library's.  Every
 * replica evolves as the single box of the same flbm_params would (the same
 * noise and the same populations, bit for bit), and the results do not
 * depend on the launch shape or on whether steps replay from the CUDA graph
 * (bit for bit).
 *
 * Work decomposition: replica r is cut into items of whole x-rows of one
 * z-plane (about item_nodes nodes); all items of all replicas are split into
 * equal contiguous chunks, one per CTA of a persistent grid.  The replica
 * populations live in one device buffer, replica after replica, each in the
 * single-box layout (SoA deviation planes, AA pattern in place).  A step
 * is two launches (the step kernel and a small per-replica statistics
 * kernel that also advances a device step counter), and runs of steps are
 * replayed from a captured CUDA graph. */
typedef struct flbm_ensemble flbm_ensemble;   /* opaque, owned by the library */

/* Launch shape of the ensemble step kernel. */
typedef struct flbm_ensemble_tuning {
    int32_t item_nodes;     /* target nodes per work item, 32..4096: rows per
                               item = the largest divisor of ny with
                               rows * nx <= max(item_nodes, nx) */
    int32_t stages;         /* items in flight per CTA (shared-memory stages), 2..4 */
    int32_t compute_warps;  /* collision warps per CTA, 1..8 (plus one copy warp) */
    int32_t ctas_per_sm;    /* resident CTAs per SM, >= 1; capped by occupancy, and
                               flbm_ensemble_get_tuning reports the granted value */
    double ms_per_step;     /* flbm_ensemble_autotune: measured time of the shape;
                               otherwise 0 */
} flbm_ensemble_tuning;

/* Create an ensemble of `count` replicas, params[r] describing replica r.
 * All replicas share scheme, precision (FLBM_FP32 or FLBM_FP16; FLBM_FP64
 * gives FLBM_E_UNSUPPORTED), stats_every and seed (one Philox key) and have
 * pairwise distinct noise_stream values, so their noise is independent;
 * tau, kT, rho0, noise_rho0 and the box may differ.  Each nx must be a
 * multiple of 32 (16-byte bulk copies) with 54 nx element bytes <= 200 KiB,
 * and N < 2^31.  State f_i = w_i rho0 at step 0.  cuda_stream: NULL for a
 * library-owned stream, else a cudaStream_t of the current device (not the
 * legacy default stream).  Default launch shape: item_nodes 256, stages 2,
 * compute_warps 8, ctas_per_sm 2. */
int flbm_ensemble_create(const flbm_params *params, int count, void *cuda_stream,
                         flbm_ensemble **out);

/* Borrowed context of replica `index` (valid until flbm_ensemble_destroy):
 * every read call of flbm_ctx works on it (moments, stats, structure factor,
 * populations, probe, state, params, step).  flbm_step and flbm_set_step on
 * it give FLBM_E_INVALID; its state may be replaced (set_populations,
 * set_state, init_thermal) only at an even ensemble step. */
int flbm_ensemble_replica(flbm_ensemble *e, int index, flbm_ctx **out);

/* Advance every replica by n >= 0 steps; returns after they completed.
 * Runs of whole graph periods (2 steps, or lcm(2, stats_every) <= 64) are
 * replayed from a CUDA graph when graphs are enabled.  FLBM_E_UNSTABLE names
 * the first failing replica; FLBM_E_TIMEOUT as for flbm_step. */
int flbm_ensemble_step(flbm_ensemble *e, int64_t n);

/* Use (1, default) or bypass (0) the CUDA graph in flbm_ensemble_step. */
int flbm_ensemble_graph(flbm_ensemble *e, int enable);

/* Set / read the launch shape.  FLBM_E_INVALID if it does not fit the
 * device (shared memory, occupancy) or is out of range. */
int flbm_ensemble_set_tuning(flbm_ensemble *e, const flbm_ensemble_tuning *t);
int flbm_ensemble_get_tuning(const flbm_ensemble *e, flbm_ensemble_tuning *out);

/* Time every valid shape of item_nodes {128, 256, 512} x stages {2, 3, 4} x
 * compute_warps {4, 8} x ctas_per_sm {1, 2} over steps_per_trial >= 1 steps
 * (after 2 warm-up steps) and keep the fastest (written to *best if not
 * NULL).  Only at step 0 (FLBM_E_INVALID otherwise); the trials advance the
 * replicas, so afterwards every replica is reset to f_i = w_i rho0, the
 * statistics are cleared and the step counter is 0 again.  Results never
 * depend on the launch shape. */
int flbm_ensemble_autotune(flbm_ensemble *e, int steps_per_trial, flbm_ensemble_tuning *best);

int flbm_ensemble_count(const flbm_ensemble *e);        /* replicas; -1 on NULL */
int64_t flbm_ensemble_get_step(const flbm_ensemble *e); /* -1 on NULL */

/* Error text of the last failing call on e; e == NULL gives the thread's
 * last create-time error. */
const char *flbm_ensemble_last_error(const flbm_ensemble *e);

/* Release the ensemble and its replica contexts (not a caller stream). */
void flbm_ensemble_destroy(flbm_ensemble *e);

/* ------------------------------------------------------------------------
 * Learned collision: a per-node network that corrects the GMF collision
 * towards the regularized collision (Reg-FLBM, Sec. III).  The paper has no
 * network; this is the library's.
 *
 *   x   28 features: the pre-collision deviations g_i = f_i - w_i rho0 in
 *       units of sqrt(rho0 kT w_i / c_s^2) (i = 0..26, ABI velocity order),
 *       and omega - 1;
 *   y   = W3 h2 + b3, h2 = silu(W2 h1 + b2), h1 = silu(W1 x + b1)
 *       (28-64-64-27, silu(z) = z / (1 + e^-z));
 *   the step adds P(w_i sigma^3 y_i), sigma = sqrt(kT / rho0), to the GMF
 *   post-collision populations, P removing mass and momentum exactly:
 *   P(d)_i = d_i - w_i (sum_j d_j + c_i . sum_j d_j c_j / c_s^2).
 *
 * Parameters: FLBM_MLP_NPARAM floats in the order W1[64][28], b1[64],
 * W2[64][64], b2[64], W3[27][64], b3[27] (row-major, W[out][in]).  The
 * tensor-core path rounds the weights, the features and both hidden
 * activations to bfloat16 (nearest, ties to even) and accumulates in FP32
 * in tensor memory; the biases stay FP32. */
#define FLBM_MLP_NPARAM 7771

/* Network outputs y[n][27] of features x[n][28] (host arrays), evaluated
 * by the tcgen05 tensor-core kernel the learned step uses.  Allocates and
 * frees its own device buffers; synchronous.  Errors via
 * flbm_last_error(NULL). */
int flbm_mlp_infer(const float *params, const float *x, int64_t n, float *y);

/* Training pairs of every node of the context's current state, written to
 * caller-owned device arrays: dev_x[N][28] features (as above, with the
 * context's rho0, kT, tau) and dev_t[N][27] targets
 *   t_i = w_i sum_{k >= 10} e_ki rho u^(deg k) / b_k / (w_i sigma^3),
 * the ghost equilibrium content by which the regularized collision
 * (Reg-FLBM, this library's reading: unit ghost relaxation towards the
 * full-order equilibrium) differs from the GMF collision of the same
 * pre-collision state, in units of the network output.  Computed in FP64,
 * stored as FP32.  Needs kT > 0.  Node n = x + nx (y + ny z).  Host
 * pointers are rejected with FLBM_E_INVALID (as by flbm_mlp_grad/train). */
int flbm_mlp_pairs(flbm_ctx *c, float *dev_x, float *dev_t);

/* Gradient of L = mean over the n samples and 27 outputs of (y - t)^2 with
 * respect to the FLBM_MLP_NPARAM parameters (FP32 forward and backward on
 * the CUDA cores, exact silu, FP64 sums over samples in a fixed order):
 * dev_x[n][28], dev_t[n][27] device arrays, grad[FLBM_MLP_NPARAM] and *loss
 * (may be NULL) host outputs.  1 <= n < 2^32.  Errors via
 * flbm_last_error(NULL). */
int flbm_mlp_grad(const float *params, const float *dev_x, const float *dev_t, int64_t n, float *grad,
                  double *loss);

/* Adam training of params (host, in place) on n device samples: `epochs`
 * passes, each over all samples in a fresh order (an affine bijection of
 * [0, n) drawn from seed), in mini-batches of `batch`; step size lr with a
 * cosine decay to 5 % over the run; beta1 0.9, beta2 0.999, eps 1e-8.
 * epoch_loss[epochs] (may be NULL) receives each epoch's mean loss over its
 * mini-batches (measured before each update). */
int flbm_mlp_train(float *params, const float *dev_x, const float *dev_t, int64_t n, int epochs, int batch,
                   double lr, uint64_t seed, double *epoch_loss);

/* Network of a FLBM_LEARNED context (FLBM_MLP_NPARAM floats, copied; may be
 * replaced between steps).  Each step then collides every node with the GMF
 * collision (noise included) and adds P(w_i sigma^3 y_i(x)) computed on the
 * tensor cores from the node's pre-collision features.  FLBM_E_INVALID for
 * other schemes. */
int flbm_set_mlp(flbm_ctx *c, const float *params);

#ifdef __cplusplus
}
#endif
#endif /* FLBM_H */
