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
    uint64_t ns;                  // slab stride: population slot i of node n at g[i * ns + n]
    uint64_t nchunks;             // cpr * ny * nz
    uint64_t step;                // t of this collision (noise counter)
    uint32_t rk[20];              // Philox round keys (k0, k1) of rounds 0..9
    uint32_t ctr2;                // noise stream id << 8 (Philox counter word 2 = block | ctr2)
    // Philox rounds 0-1 of the launch-uniform counter words (step, block |
    // ctr2) for blocks 0..5, precomputed on the host (philox4x32_10_r2)
    uint32_t ph_zk;               // step hi ^ rk[1]
    uint32_t ph_u1[6], ph_u2[6], ph_u3[6];
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

// ---------------------------------------------------------------------------
// Batched ensemble (ens_kernel.cuh): many independent periodic boxes advanced
// by one persistent kernel.  Each replica is cut into work items of rpi whole
// x-rows of one z-plane (rpi divides ny); the items of all replicas form one
// global sequence that the CTAs split into contiguous, equal-length chunks.

// One replica, as the kernels see it (device table, host-built).
struct EnsReplica {
    void *g;                      // its deviation planes g[i*n + node]
    uint64_t n;                   // nodes
    uint64_t item0;               // global index of its first item
    uint32_t nx, ny, nz;
    uint32_t rpi;                 // x-rows per item (divides ny)
    uint32_t item_nodes;          // rpi * nx
    uint32_t items_per_plane;     // ny / rpi
    uint32_t ctr2;                // noise stream << 8
    int32_t noise_rho0;
    double rho0, sqrt_rho0;       // the scalars of StepArgs, per replica
    double lambda, omega, amp_h, amp_g;
    int32_t cta_lo, cta_hi;       // CTAs whose chunks meet this replica
    DevStats *st;                 // accumulators of the replica's context
    unsigned long long *bad_step; // first unstable step of this replica
};

struct EnsArgs {
    uint32_t rk[20];              // Philox round keys (one key for the ensemble)
    const EnsReplica *reps;
    uint32_t nrep;
    uint32_t stages;              // shared-memory stages per CTA (2..kEnsMaxStages)
    uint32_t stride;              // elements per staged segment (>= every item_nodes)
    uint32_t tx_pad;              // failure injection (0 normally)
    uint64_t nitems;              // items of all replicas
    const unsigned long long *dstep;   // t of this step (advanced by the post kernel)
    double *partials;             // [grid + nrep][NSTAT]: slot (cta + replica)
    unsigned int *flag;           // bit 0: instability; bit 1: a bounded wait ran out
};
constexpr int kEnsMaxStages = 4;
constexpr int kEnsMaxWarps = 8;    // compute warps per CTA at most

// Chunk [begin, end) of the global item sequence owned by CTA b of grid.
__host__ __device__ inline void ens_chunk(uint64_t nitems, uint32_t b, uint32_t grid, uint64_t &begin,
                                          uint64_t &end)
{
    const uint64_t k = nitems / grid, rem = nitems % grid;
    begin = uint64_t(b) * k + (uint64_t(b) < rem ? uint64_t(b) : rem);
    end = begin + k + (uint64_t(b) < rem ? 1u : 0u);
}

// Launchers (ens_f32.cu, ens_f16.cu; the two-node kernels in ens_f32p.cu,
// ens_f16p.cu): the step kernel with np nodes per compute thread, `threads`
// threads (compute warps + one copy warp) and `smem` dynamic shared bytes,
// and its resident CTAs per SM (0 if the shape does not fit; also sets the
// kernels' shared-memory attribute on the current device).
cudaError_t launch_ens_step_f32(const EnsArgs &a, int scheme, bool odd, bool stats, int grid,
                                int threads, size_t smem, cudaStream_t s, int np);
cudaError_t launch_ens_step_f16(const EnsArgs &a, int scheme, bool odd, bool stats, int grid,
                                int threads, size_t smem, cudaStream_t s, int np);
int ens_occupancy_f32(int scheme, int threads, size_t smem, int np);
int ens_occupancy_f16(int scheme, int threads, size_t smem, int np);
cudaError_t launch_ens_step_f32p(const EnsArgs &a, int scheme, bool odd, bool stats, int grid,
                                 int threads, size_t smem, cudaStream_t s);
cudaError_t launch_ens_step_f16p(const EnsArgs &a, int scheme, bool odd, bool stats, int grid,
                                 int threads, size_t smem, cudaStream_t s);
int ens_occupancy_f32p(int scheme, int threads, size_t smem);
int ens_occupancy_f16p(int scheme, int threads, size_t smem);
// Whether the two-node row and ensemble kernels serve FP32 / FP16 storage:
// FLBM_ROW_PAIRS=0 (environment, read at every call) keeps one node per
// thread (a measuring knob; the default is two).  Both give the same bits.
bool row_pairs_enabled();
// After each ensemble step: per-replica FP64 totals of the partial slots into
// each replica's DevStats (stats steps), then the step counter advances.
cudaError_t launch_ens_post(const EnsArgs &a, bool stats, uint32_t cwarps, unsigned int *done,
                            unsigned long long *dstep, cudaStream_t s);

// Step-kernel launchers (step_f64.cu, step_f32.cu).  grid: CTAs of the
// direct kernel; row_grid: CTAs of the TMA row pipeline (0: do not use it).
cudaError_t launch_step_f64(double *g, const StepArgs<double> &a, int scheme, bool odd,
                            bool stats, int grid, int row_grid, cudaStream_t s);
cudaError_t launch_step_f32(float *g, const StepArgs<float> &a, int scheme, bool odd,
                            bool stats, int grid, int row_grid, cudaStream_t s);
cudaError_t launch_step_f16(void *g, const StepArgs<float> &a, int scheme, bool odd,
                            bool stats, int grid, int row_grid, cudaStream_t s);
// Resident CTAs per SM of the direct kernel and of the row pipeline (0 when
// it does not serve rows of length nx) for (precision, scheme, stats; ns, the
// slab stride, picks the index width); also
// prepares the kernels' shared-memory attributes on the current device.
void step_occupancy_f64(int scheme, uint32_t nx, bool stats, int &direct, int &rows);
void step_occupancy_f32(int scheme, uint32_t nx, uint64_t ns, bool stats, int &direct, int &rows);
void step_occupancy_f16(int scheme, uint32_t nx, uint64_t ns, bool stats, int &direct, int &rows);
// The FP16-storage two-node row kernels for rows of exactly 512 nodes
// (step_f16_nx512.cu), which step_f16.cu calls when the row plan of the box
// takes two nodes per thread in full CTAs.  FP32 keeps the general kernel:
// there the step is at the HBM bound and the fixed length gains nothing.
cudaError_t launch_rows_f16_nx512(void *g, const StepArgs<float> &a, int scheme, bool odd, bool stats,
                                  int row_grid, cudaStream_t s);
int rows_occupancy_f16_nx512(int scheme, bool stats);
// The PACED FP32 two-node row kernels (step_f32_paced.cu) for rows staged
// twice, which step_f32.cu calls when rows_paced<float> holds for the box.
cudaError_t launch_rows_f32_paced(float *g, const StepArgs<float> &a, int scheme, bool odd, bool stats,
                                  int row_grid, cudaStream_t s);
int rows_occupancy_f32_paced(int scheme, bool stats, uint32_t nx);

// Step constants shared by flbm_step and flbm_step_noalloc (capi.cu): the
// Philox round keys, the density used by the noise, and the per-mode
// relaxation / equilibrium / noise coefficients of the scheme.
// Grids of the direct step kernel and of the row pipeline (0: not used) for
// a box on nsm SMs, given the kernels' resident CTAs per SM; honours the
// FLBM_CTAS_PER_SM and FLBM_ROWS=0 environment knobs.
void step_grids(const flbm_params &p, int nsm, int occ, int occ_rows, int &grid, int &row_grid);
void fill_step_constants(const flbm_params &p, StepArgs<float> &a);
void fill_step_constants(const flbm_params &p, StepArgs<double> &a);
// Set the calling thread's error text returned by flbm_last_error(NULL).
void set_thread_error(const char *msg);
}  // namespace flbm

#include <vector>

namespace flbm {
// Moment-state form (mstate.cu): ten FP32 numbers per node between steps,
// kMsVals arrays of N: rho - rho0, j_x, j_y, j_z, Q_xx, Q_yy, Q_zz, Q_xy,
// Q_xz, Q_yz.  ms_prepare sets the kernels' shared-memory attribute and
// picks the grid and the z-segment length; the noise arguments an name step
// t - 1, the collision arguments ac step t.
constexpr int kMsVals = 10;
cudaError_t ms_prepare(int scheme, int nsm, const StepArgs<float> &a, int &grid, int &zseg);
cudaError_t launch_ms_boot(const float *g, float *ms, const StepArgs<float> &a, int scheme, bool odd, bool stats,
                           int grid, cudaStream_t s);
cudaError_t launch_ms_step(const float *ms_in, float *ms_out, const StepArgs<float> &an, const StepArgs<float> &ac,
                           int scheme, bool stats, int grid, int zseg, cudaStream_t s);
cudaError_t launch_ms_export(const float *ms, float *g, const StepArgs<float> &an, int scheme, int grid, int zseg,
                             cudaStream_t s);
// Learned-collision network: the bf16 image of weights and split biases in
// the tensor-core operand layout (mlp_tc.cuh, mlp_infer.cu) from the flat
// FP32 parameter vector of include/flbm.h (FLBM_MLP_NPARAM values).
void build_mlp_image(const float *params, std::vector<unsigned char> &img);
// The learned step (step_learned.cu): GMF collision + network correction.
struct LearnArgs {
    const unsigned char *img;   // network image (build_mlp_image), device
    float inv_s[4];             // 1 / sqrt(rho0 kT w / c_s^2) for |c|^2 = 0, 1, 2, 3
    float sig3;                 // (kT / rho0)^(3/2)
    float x27;                  // omega - 1
    int32_t starve;             // failure injection (tests): never commit layer 1
};
cudaError_t launch_step_learned(float *g, const StepArgs<float> &a, const LearnArgs &L, bool odd, bool stats,
                                int grid, cudaStream_t s);
// Resident CTAs per SM of the learned step (1: a CTA holds all of an SM's
// tensor memory); also sets the kernels' shared-memory attribute.
int learned_occupancy(uint64_t n);
// Training pairs (mlp_train.cu) of cn nodes from FP64 deviations g[27][cn]:
// features X[cn][28] and targets T[cn][27] (device arrays).
cudaError_t launch_mlp_pairs(const double *g, uint64_t cn, double rho0, double kT, double omega, float *X,
                             float *T, cudaStream_t s);

// Auxiliary kernels (aux.cu).  `prec` is 0 (double storage), 1 (float) or
// 2 (half).
struct BoxDesc {
    uint32_t nx, ny, nz;
    uint64_t n;
    uint64_t ns;           // slab stride of the population storage (>= n)
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
