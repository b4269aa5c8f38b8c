// ctx.h -- the context behind flbm_ctx, shared by capi.cu (one box) and
// ensemble.cu (a batch of boxes whose contexts are views into one buffer).
#pragma once

#include <cufft.h>

#include <string>
#include <vector>

#include "../../include/flbm.h"
#include "internal.h"

namespace flbm {

struct DevFlags {
    unsigned int flag;
    unsigned int pad;
    unsigned long long bad_step;
};

}  // namespace flbm

struct flbm_ctx {
    flbm_params p{};
    int device = 0;
    int nsm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *g = nullptr;
    bool own_g = false;
    size_t g_bytes = 0;
    uint64_t n = 0;
    uint64_t ns = 0;               // slab stride: population slot i of node n at g[i * ns + n]
    int64_t step = 0;
    int phase = 0;                 // storage is natural when ((step + phase) & 1) == 0
    uint32_t tx_pad = 0;           // failure injection into the row pipeline (tests)
    int grid = 1;                  // persistent grid of the direct step kernel
    int row_grid = 0;              // persistent grid of the TMA row pipeline (0: unused)
    double *partials = nullptr;    // [max(grid, row_grid)][NSTAT]
    flbm::DevStats *dstats = nullptr;
    flbm::DevFlags *dflags = nullptr;
    // host transfers: two staging buffers of pipe_nodes * 27 doubles, a copy
    // stream, and events that hand each buffer between the streams
    double *pipe[2] = {nullptr, nullptr};
    uint64_t pipe_nodes = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_ready[2] = {nullptr, nullptr};
    cudaEvent_t ev_free[2] = {nullptr, nullptr};
    // S(k)
    cufftHandle plan = 0;
    bool has_plan = false;
    void *fft_in = nullptr;
    void *fft_out = nullptr;
    double *shell_s = nullptr;
    unsigned long long *shell_c = nullptr;
    int shell_cap = 0;
    // step-kernel timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;   // pairs (start, stop), reused
    size_t ev_used = 0;            // pairs recorded since the last read
    // replica of an ensemble: stepped only through the ensemble, destroyed
    // with it; its state may be replaced only while the ensemble's storage
    // is in the natural form
    flbm_ensemble *ens = nullptr;
    // FLBM_LEARNED: the network image on the device (flbm_set_mlp)
    unsigned char *mlp_img = nullptr;
    // FLBM_STATE_MOMENTS: two arrays of kMsVals * n floats; ms[ms_cur] holds
    // the state of collision step - 1 while ms_live; the populations in g
    // are current while pops_valid (at least one of the two holds)
    float *ms[2] = {nullptr, nullptr};
    int ms_cur = 0;
    bool ms_live = false;
    bool pops_valid = true;
    int ms_grid = 1;               // CTAs of the moment-state step (one per SM)
    int ms_zseg = 1;               // z planes a CTA marches per work item
    std::string err;
};

namespace flbm {

// Parameter check shared by every creation path ("" when valid).
std::string validate_params(const flbm_params *p);
// Context creation / destruction (capi.cu).
int create_ctx(const flbm_params *p, void *dev_buf, size_t dev_bytes, void *stream, flbm_ctx **out);
void destroy_ctx(flbm_ctx *c);
// A replica's state was replaced: clear the ensemble's sticky failure flags
// (ensemble.cu).
void ensemble_state_replaced(flbm_ensemble *e);

}  // namespace flbm
