// internal.h -- structures shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

struct flbm_params;

namespace flbm {

constexpr int kQ = 27;
constexpr int NSTAT = 13;     // fused reduction slots, see StatSlot
constexpr int kBlock = 128;   // threads per CTA of the step kernel (one x-row chunk)

// Minimum resident CTAs per SM requested from the compiler for the step
// kernel (bounds its registers per thread); a build option.
#ifndef FLBM_MIN_BLOCKS
#define FLBM_MIN_BLOCKS 4
#endif
// Slots of the fused FP64 reductions (row a9).  Sums over nodes of the
// pre-collision state: drho = rho - rho0, j, u^2 and the four
// equilibration-ratio observables m1 = drho, m2 = sum_a j_a (its sum is
// S_JX + S_JY + S_JZ), m3 = sum_a Pi_aa - rho0, m4 = sum_{a<b} Pi_ab, and
// their squares.
enum StatSlot {
    S_DRHO = 0, S_JX, S_JY, S_JZ, S_UX2, S_UY2, S_UZ2,
    S_M3, S_M4, S_M1SQ, S_M2SQ, S_M3SQ, S_M4SQ
};

template <typename R>
struct StepArgs {
    uint32_t nx, ny, nz, cpr;     // box; x-chunks of kBlock nodes per row
    uint64_t n;                   // nodes
    uint64_t nchunks;             // cpr * ny * nz
    uint64_t step;                // t of this collision (noise counter)
    uint32_t rk[20];              // Philox round keys (k0, k1) of rounds 0..9
    int32_t noise_rho0;           // phi_k uses rho0 instead of rho(x,t)
    uint32_t tx_pad;              // failure injection: bytes the row pipeline
                                  // expects beyond what it copies (0 normally)
    R rho0;
    R sqrt_rho0;
    // Relaxation and noise scalars; the per-mode factors (syn_scale,
    // fwd_scale, sqrt(b_k / c_s^2)) are compile-time constants of the kernel.
    R lambda;                     // 1 - omega: k = 4..9, and every k for BGK-FLBM
    R omega;                      // weight of the equilibrium in k = 4..9
    R amp_h;                      // sqrt(kT omega (2 - omega)), Eq. fluct_phi
    R amp_g;                      // ghosts: sqrt(kT) (Eq. fluct_phig), amp_h for BGK
    double *partials;             // [gridDim.x][NSTAT] when reducing
    unsigned int *flag;           // bit 0: instability; bit 1: a bounded wait ran out
    unsigned long long *bad_step; // first step that met rho <= 0 / non-finite
};

// Device-side accumulators of the fused reductions.
struct DevStats {
    double last[NSTAT];    // global sums of the most recent reduced step
    double acc_u2[3];      // sum over reduced steps of mean_x u_a^2
    double acc_m[4];       // sum over reduced steps of mean_x m_k
    double acc_m2[4];      // sum over reduced steps of mean_x m_k^2
    long long step;        // t of the most recent reduced step
    long long nsamp;       // reduced steps since reset
};

// Step-kernel launchers (step_f64.cu, step_f32.cu).  grid: CTAs of the
// direct kernel; row_grid: CTAs of the TMA row pipeline (0: do not use it).
cudaError_t launch_step_f64(double *g, const StepArgs<double> &a, int scheme, bool odd,
                            bool stats, int grid, int row_grid, cudaStream_t s);
cudaError_t launch_step_f32(float *g, const StepArgs<float> &a, int scheme, bool odd,
                            bool stats, int grid, int row_grid, cudaStream_t s);
cudaError_t launch_step_f16(void *g, const StepArgs<float> &a, int scheme, bool odd,
                            bool stats, int grid, int row_grid, cudaStream_t s);
// Resident CTAs per SM of the direct kernel and of the row pipeline (0 when
// it does not serve rows of length nx) for (precision, scheme, stats); also
// prepares the kernels' shared-memory attributes on the current device.
void step_occupancy_f64(int scheme, uint32_t nx, bool stats, int &direct, int &rows);
void step_occupancy_f32(int scheme, uint32_t nx, uint64_t n, bool stats, int &direct, int &rows);
void step_occupancy_f16(int scheme, uint32_t nx, uint64_t n, bool stats, int &direct, int &rows);

// Step constants shared by flbm_step and flbm_step_noalloc (capi.cu): the
// Philox round keys, the density used by the noise, and the per-mode
// relaxation / equilibrium / noise coefficients of the scheme.
void fill_step_constants(const flbm_params &p, StepArgs<float> &a);
void fill_step_constants(const flbm_params &p, StepArgs<double> &a);
// Set the calling thread's error text returned by flbm_last_error(NULL).
void set_thread_error(const char *msg);

// Auxiliary kernels (aux.cu).  `prec` is 0 (double storage), 1 (float) or
// 2 (half).
struct BoxDesc {
    uint32_t nx, ny, nz;
    uint64_t n;
    double rho0;
    int parity;            // 0: storage natural; 1: AA-shifted (odd form)
};
cudaError_t launch_fill_rest(void *g, int prec, uint64_t count, cudaStream_t s);
cudaError_t launch_gather_f(const void *g, int prec, const BoxDesc &b, uint64_t n0, uint64_t cn,
                            double *out, bool deviations, cudaStream_t s);
cudaError_t launch_gather_state(const void *g, int prec, const BoxDesc &b, uint64_t n0,
                                uint64_t cn, void *out, cudaStream_t s);
cudaError_t launch_scatter_f(void *g, int prec, const BoxDesc &b, uint64_t n0, uint64_t cn,
                             const double *in, cudaStream_t s);
cudaError_t launch_init_thermal(void *g, int prec, const BoxDesc &b, double kT, uint64_t seed,
                                cudaStream_t s);
cudaError_t launch_probe(const void *g, int prec, const BoxDesc &b, const long long *nodes,
                         long long count, double *out, cudaStream_t s);
cudaError_t launch_moments(const void *g, int prec, const BoxDesc &b, uint64_t n0, uint64_t cn,
                           double *out, cudaStream_t s);
cudaError_t launch_observable(const void *g, int prec, const BoxDesc &b, int obs, void *field,
                              cudaStream_t s);
cudaError_t launch_shells(const void *spec, int prec, const BoxDesc &b, int nshell, double *S,
                          unsigned long long *cnt, cudaStream_t s);
cudaError_t launch_stats_finalize(const double *partials, int nblocks, DevStats *st,
                                  long long step, double n, cudaStream_t s);

}  // namespace flbm
