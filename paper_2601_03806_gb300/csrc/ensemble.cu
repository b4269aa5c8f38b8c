// ensemble.cu -- host side of the batched ensemble (flbm_ensemble_* in
// include/flbm.h): replica contexts as views into one device buffer, the
// work-item table, the launch shape and its autotuner, and CUDA-graph
// replay of whole step periods.  The arithmetic runs in ens_kernel.cuh.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/flbm.h"
#include "ctx.h"
#include "internal.h"

using namespace flbm;

namespace {

thread_local std::string g_ens_error;

constexpr int kMaxGraphPeriod = 64;            // steps in one captured graph at most
constexpr size_t kMaxStageBytes = 200 * 1024;  // dynamic shared memory of a CTA at most

}  // namespace

struct flbm_ensemble {
    int nrep = 0;
    flbm_params p0{};                   // shared fields: scheme, precision, stats_every, seed
    int device = 0;
    int nsm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *g = nullptr;
    size_t g_bytes = 0;
    std::vector<flbm_ctx *> reps;
    std::vector<size_t> offsets;        // byte offset of each replica in g
    std::vector<EnsReplica> htab;
    EnsReplica *dtab = nullptr;
    double *partials = nullptr;
    size_t partial_elems = 0;
    // device bookkeeping: [0] step counter, [1] post-kernel arrivals (low
    // word), [2] failure flag (low word), then bad_step per replica
    unsigned long long *dbook = nullptr;
    EnsArgs args{};
    flbm_ensemble_tuning tune{};
    int grid = 0;
    int threads = 0;
    size_t smem = 0;
    int np = 1;                        // nodes per compute thread of the step kernel
    int64_t step = 0;
    bool use_graph = true;
    cudaGraphExec_t gexec = nullptr;
    uint32_t tx_pad = 0;
    std::string err;

    unsigned long long *dstep() { return dbook; }
    unsigned int *done() { return reinterpret_cast<unsigned int *>(dbook + 1); }
    unsigned int *flag() { return reinterpret_cast<unsigned int *>(dbook + 2); }
    unsigned long long *bad_steps() { return dbook + 3; }
};

namespace {

int efail(flbm_ensemble *e, int code, const std::string &msg)
{
    if (e) e->err = msg;
    else g_ens_error = msg;
    return code;
}

#define ECK(e, call)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return efail(e, FLBM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

size_t elem_bytes(int prec) { return prec == FLBM_FP16 ? 2 : 4; }

int occupancy(const flbm_ensemble *e, int threads, size_t smem)
{
    return e->p0.precision == FLBM_FP32 ? ens_occupancy_f32(e->p0.scheme, threads, smem, e->np)
                                        : ens_occupancy_f16(e->p0.scheme, threads, smem, e->np);
}

std::string validate_ensemble(const flbm_params *params, int count)
{
    if (!params) return "params is NULL";
    if (count < 1 || count > (1 << 16)) return "count must be in [1, 65536]";
    const flbm_params &p0 = params[0];
    std::vector<int32_t> streams;
    for (int r = 0; r < count; ++r) {
        const flbm_params &p = params[r];
        const std::string why = validate_params(&p);
        if (!why.empty()) return "replica " + std::to_string(r) + ": " + why;
        if (p.scheme != p0.scheme || p.precision != p0.precision || p.stats_every != p0.stats_every ||
            p.seed != p0.seed)
            return "replica " + std::to_string(r) +
                   ": scheme, precision, stats_every and seed must match replica 0";
        if (p.scheme > FLBM_REG) return "replica " + std::to_string(r) + ": the ensemble runs BGK, GMF or Reg";
        if (p.state_form != FLBM_STATE_POPULATIONS)
            return "replica " + std::to_string(r) + ": the ensemble keeps populations (state_form 0)";
        if (p.nx % 32 != 0) return "replica " + std::to_string(r) + ": nx must be a multiple of 32";
        if (size_t(2) * kQ * size_t(p.nx) * elem_bytes(p.precision) > kMaxStageBytes)
            return "replica " + std::to_string(r) + ": nx too large for two shared-memory stages";
        if (uint64_t(p.nx) * uint64_t(p.ny) * uint64_t(p.nz) >= (1ull << 31))
            return "replica " + std::to_string(r) + ": N must be < 2^31";
        streams.push_back(p.noise_stream);
    }
    std::sort(streams.begin(), streams.end());
    if (std::adjacent_find(streams.begin(), streams.end()) != streams.end())
        return "noise_stream values must be pairwise distinct";
    return "";
}

// Build the item table for tuning t and upload it; sets the launch shape.
int apply_tuning(flbm_ensemble *e, const flbm_ensemble_tuning &t)
{
    if (t.item_nodes < 32 || t.item_nodes > 4096 || t.stages < 2 || t.stages > kEnsMaxStages ||
        t.compute_warps < 1 || t.compute_warps > kEnsMaxWarps || t.ctas_per_sm < 1)
        return efail(e, FLBM_E_INVALID, "tuning out of range");
    std::vector<EnsReplica> tab(e->htab);
    uint64_t item0 = 0;
    uint32_t stride = 0;
    for (int r = 0; r < e->nrep; ++r) {
        EnsReplica &rp = tab[r];
        const uint32_t cap = std::max<uint32_t>(uint32_t(t.item_nodes), rp.nx) / rp.nx;
        uint32_t rpi = 1;
        for (uint32_t k = 1; k <= std::min(cap, rp.ny); ++k)
            if (rp.ny % k == 0) rpi = k;
        rp.rpi = rpi;
        rp.item_nodes = rpi * rp.nx;
        rp.items_per_plane = rp.ny / rpi;
        rp.item0 = item0;
        item0 += uint64_t(rp.items_per_plane) * rp.nz;
        stride = std::max(stride, rp.item_nodes);
    }
    const uint64_t nitems = item0;
    const size_t smem = size_t(t.stages) * kQ * stride * elem_bytes(e->p0.precision);
    if (smem > kMaxStageBytes) return efail(e, FLBM_E_INVALID, "tuning needs too much shared memory");
    const int threads = t.compute_warps * 32 + 32;
    // two adjacent nodes per compute thread (packed FP32 pairs) unless
    // FLBM_ROW_PAIRS=0; the same bits either way
    e->np = row_pairs_enabled() ? 2 : 1;
    const int occ = occupancy(e, threads, smem);
    if (occ < 1) return efail(e, FLBM_E_INVALID, "tuning does not fit the device");
    const int per_sm = std::min(occ, int(t.ctas_per_sm));
    const int grid = int(std::max<uint64_t>(1, std::min<uint64_t>(nitems, uint64_t(e->nsm) * per_sm)));
    // CTAs whose chunks meet each replica
    for (int r = 0; r < e->nrep; ++r) {
        EnsReplica &rp = tab[r];
        const uint64_t first = rp.item0, last = rp.item0 + uint64_t(rp.items_per_plane) * rp.nz - 1;
        auto owner = [&](uint64_t i) {
            int lo = 0, hi = grid - 1;   // largest b with begin(b) <= i
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                uint64_t b0, b1;
                ens_chunk(nitems, uint32_t(mid), uint32_t(grid), b0, b1);
                if (b0 <= i) lo = mid;
                else hi = mid - 1;
            }
            return lo;
        };
        rp.cta_lo = owner(first);
        rp.cta_hi = owner(last);
    }
    const size_t need = (size_t(grid) + e->nrep) * kEnsMaxWarps * NSTAT;
    if (need > e->partial_elems) {
        cudaFree(e->partials);
        e->partials = nullptr;
        e->partial_elems = 0;
        ECK(e, cudaMalloc(&e->partials, need * sizeof(double)));
        e->partial_elems = need;
    }
    ECK(e, cudaMemcpyAsync(e->dtab, tab.data(), tab.size() * sizeof(EnsReplica), cudaMemcpyHostToDevice,
                           e->stream));
    ECK(e, cudaStreamSynchronize(e->stream));
    e->htab = tab;
    e->args.stages = uint32_t(t.stages);
    e->args.stride = stride;
    e->args.nitems = nitems;
    e->args.partials = e->partials;
    e->tune = t;
    e->tune.ctas_per_sm = per_sm;      // what the device grants, not what was asked
    e->tune.ms_per_step = 0.0;
    e->grid = grid;
    e->threads = threads;
    e->smem = smem;
    if (e->gexec) {
        cudaGraphExecDestroy(e->gexec);
        e->gexec = nullptr;
    }
    return FLBM_OK;
}

int graph_period(const flbm_ensemble *e)
{
    const int every = e->p0.stats_every;
    if (every <= 0) return 2;
    return every % 2 == 0 ? every : 2 * every;
}

cudaError_t launch_one(flbm_ensemble *e, int64_t t)
{
    const bool odd = (t & 1) != 0;   // every replica shares the AA parity; phase 0
    const int every = e->p0.stats_every;
    const bool stats = every > 0 && t % every == 0;
    cudaError_t err = e->p0.precision == FLBM_FP32
        ? launch_ens_step_f32(e->args, e->p0.scheme, odd, stats, e->grid, e->threads, e->smem, e->stream, e->np)
        : launch_ens_step_f16(e->args, e->p0.scheme, odd, stats, e->grid, e->threads, e->smem, e->stream, e->np);
    if (err != cudaSuccess) return err;
    return launch_ens_post(e->args, stats, uint32_t(e->tune.compute_warps), e->done(), e->dstep(), e->stream);
}

// Capture one graph period starting at a step t0 with t0 % period == 0.
int build_graph(flbm_ensemble *e, int64_t t0, int period)
{
    cudaGraph_t graph = nullptr;
    ECK(e, cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < period && err == cudaSuccess; ++k) err = launch_one(e, t0 + k);
    cudaError_t end = cudaStreamEndCapture(e->stream, &graph);
    if (err != cudaSuccess || end != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return efail(e, FLBM_E_CUDA, std::string("graph capture: ") +
                                         cudaGetErrorString(err != cudaSuccess ? err : end));
    }
    err = cudaGraphInstantiate(&e->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) {
        e->gexec = nullptr;
        return efail(e, FLBM_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(err));
    }
    return FLBM_OK;
}

// Launch n steps from e->step (no synchronisation, no flag check).
int launch_steps(flbm_ensemble *e, int64_t n)
{
    const int period = graph_period(e);
    int64_t k = 0;
    while (k < n) {
        const int64_t t = e->step + k;
        if (e->use_graph && period <= kMaxGraphPeriod && t % period == 0 && n - k >= period) {
            if (!e->gexec) {
                const int rc = build_graph(e, t, period);
                if (rc) return rc;
            }
            for (; n - k >= period; k += period) ECK(e, cudaGraphLaunch(e->gexec, e->stream));
        } else {
            ECK(e, launch_one(e, t));
            ++k;
        }
    }
    e->step += n;
    for (flbm_ctx *c : e->reps) c->step = e->step;
    return FLBM_OK;
}

int check_flags(flbm_ensemble *e)
{
    unsigned long long book[3];
    ECK(e, cudaMemcpyAsync(book, e->dbook, sizeof(book), cudaMemcpyDeviceToHost, e->stream));
    ECK(e, cudaStreamSynchronize(e->stream));
    const unsigned int flag = unsigned(book[2] & 0xffffffffu);
    if (flag & 2u) return efail(e, FLBM_E_TIMEOUT, "a bounded device wait ran out during the last steps");
    if (flag) {
        std::vector<unsigned long long> bad(e->nrep);
        ECK(e, cudaMemcpy(bad.data(), e->bad_steps(), bad.size() * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost));
        int worst = 0;
        for (int r = 1; r < e->nrep; ++r)
            if (bad[r] < bad[worst]) worst = r;
        return efail(e, FLBM_E_UNSTABLE, "instability: rho <= 0 or non-finite in replica " +
                                             std::to_string(worst) + " at step " +
                                             std::to_string(int64_t(bad[worst])));
    }
    return FLBM_OK;
}

int reset_flags(flbm_ensemble *e)
{
    ECK(e, cudaMemsetAsync(e->dbook + 2, 0, sizeof(unsigned long long), e->stream));
    ECK(e, cudaMemsetAsync(e->bad_steps(), 0xff, size_t(e->nrep) * sizeof(unsigned long long), e->stream));
    return FLBM_OK;
}

// Back to the state of creation: f_i = w_i rho0, statistics cleared, step 0.
int reset_all(flbm_ensemble *e)
{
    const size_t es = elem_bytes(e->p0.precision);
    ECK(e, launch_fill_rest(e->g, e->p0.precision == FLBM_FP32 ? 1 : 2, e->g_bytes / es, e->stream));
    for (flbm_ctx *c : e->reps) {
        ECK(e, cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), e->stream));
        c->step = 0;
        c->phase = 0;
    }
    ECK(e, cudaMemsetAsync(e->dbook, 0, 2 * sizeof(unsigned long long), e->stream));
    int rc = reset_flags(e);
    if (rc) return rc;
    ECK(e, cudaStreamSynchronize(e->stream));
    e->step = 0;
    return FLBM_OK;
}

void release(flbm_ensemble *e)
{
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    for (flbm_ctx *c : e->reps) {
        if (!c) continue;
        c->ens = nullptr;
        destroy_ctx(c);
    }
    cudaFree(e->partials);
    cudaFree(e->dtab);
    cudaFree(e->dbook);
    cudaFree(e->g);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

}  // namespace

void flbm::ensemble_state_replaced(flbm_ensemble *e)
{
    if (!e) return;
    reset_flags(e);
    cudaStreamSynchronize(e->stream);
}

extern "C" {

int flbm_ensemble_create(const flbm_params *params, int count, void *cuda_stream, flbm_ensemble **out)
{
    if (!out) return efail(nullptr, FLBM_E_INVALID, "out is NULL");
    *out = nullptr;
    const std::string why = validate_ensemble(params, count);
    if (!why.empty()) return efail(nullptr, FLBM_E_INVALID, why);
    if (params[0].precision == FLBM_FP64)
        return efail(nullptr, FLBM_E_UNSUPPORTED, "the ensemble stores FP32 or FP16 populations");
    flbm_ensemble *e = new (std::nothrow) flbm_ensemble;
    if (!e) return efail(nullptr, FLBM_E_NOMEM, "host allocation failed");
    auto bail = [&](int code) {
        g_ens_error = e->err;
        release(e);
        return code;
    };
    e->nrep = count;
    e->p0 = params[0];
    cudaError_t err = cudaGetDevice(&e->device);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&e->nsm, cudaDevAttrMultiProcessorCount, e->device);
    if (err != cudaSuccess) {
        e->err = std::string("no usable CUDA device: ") + cudaGetErrorString(err);
        return bail(FLBM_E_CUDA);
    }
    if (cuda_stream) {
        e->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
        if (err != cudaSuccess) { e->err = cudaGetErrorString(err); return bail(FLBM_E_CUDA); }
        e->own_stream = true;
    }
    // one buffer, replica after replica, each 256-byte aligned
    const size_t es = elem_bytes(params[0].precision);
    size_t off = 0;
    for (int r = 0; r < count; ++r) {
        e->offsets.push_back(off);
        const size_t b = size_t(params[r].nx) * params[r].ny * params[r].nz * kQ * es;
        off += (b + 255) / 256 * 256;
    }
    e->g_bytes = off;
    err = cudaMalloc(&e->g, e->g_bytes);
    if (err == cudaSuccess) err = cudaMalloc(&e->dtab, size_t(count) * sizeof(EnsReplica));
    if (err == cudaSuccess) err = cudaMalloc(&e->dbook, (3 + size_t(count)) * sizeof(unsigned long long));
    if (err != cudaSuccess) {
        e->err = std::string("cudaMalloc: ") + cudaGetErrorString(err);
        return bail(FLBM_E_NOMEM);
    }
    // replica contexts: views on the shared buffer and stream
    e->reps.assign(count, nullptr);
    e->htab.resize(count);
    for (int r = 0; r < count; ++r) {
        flbm_ctx *c = nullptr;
        char *slice = static_cast<char *>(e->g) + e->offsets[r];
        const size_t bytes = size_t(params[r].nx) * params[r].ny * params[r].nz * kQ * es;
        const int rc = create_ctx(&params[r], slice, bytes, e->stream, &c);
        if (rc != FLBM_OK) {
            e->err = "replica " + std::to_string(r) + ": " + flbm_last_error(nullptr);
            return bail(rc);
        }
        c->ens = e;
        e->reps[r] = c;
        StepArgs<double> sa;
        std::memset(&sa, 0, sizeof(sa));
        fill_step_constants(params[r], sa);
        if (r == 0) std::memcpy(e->args.rk, sa.rk, sizeof(sa.rk));
        EnsReplica &rp = e->htab[r];
        std::memset(&rp, 0, sizeof(rp));
        rp.g = slice;
        rp.n = c->n;
        rp.nx = uint32_t(params[r].nx);
        rp.ny = uint32_t(params[r].ny);
        rp.nz = uint32_t(params[r].nz);
        rp.ctr2 = sa.ctr2;
        rp.noise_rho0 = sa.noise_rho0;
        rp.rho0 = sa.rho0;
        rp.sqrt_rho0 = sa.sqrt_rho0;
        rp.lambda = sa.lambda;
        rp.omega = sa.omega;
        rp.amp_h = sa.amp_h;
        rp.amp_g = sa.amp_g;
        rp.st = c->dstats;
        rp.bad_step = e->bad_steps() + r;
    }
    // FLBM_INJECT_STARVE=1 (environment, failure-injection tests only): the
    // pipeline expects 16 bytes more than it copies, so its bounded waits
    // run out and flbm_ensemble_step reports FLBM_E_TIMEOUT
    if (const char *inj = std::getenv("FLBM_INJECT_STARVE"))
        if (std::atoi(inj) == 1) e->tx_pad = 16;
    e->args.reps = e->dtab;
    e->args.nrep = uint32_t(count);
    e->args.tx_pad = e->tx_pad;
    e->args.dstep = e->dstep();
    e->args.flag = e->flag();
    flbm_ensemble_tuning t{256, 2, 8, 2, 0.0};
    int rc = apply_tuning(e, t);
    if (rc != FLBM_OK) {
        t.ctas_per_sm = 1;
        rc = apply_tuning(e, t);
    }
    if (rc != FLBM_OK) return bail(rc);
    rc = reset_all(e);
    if (rc != FLBM_OK) return bail(rc);
    *out = e;
    return FLBM_OK;
}

int flbm_ensemble_replica(flbm_ensemble *e, int index, flbm_ctx **out)
{
    if (!e || !out) return efail(e, FLBM_E_INVALID, "NULL argument");
    if (index < 0 || index >= e->nrep) return efail(e, FLBM_E_INVALID, "replica index out of range");
    *out = e->reps[index];
    return FLBM_OK;
}

int flbm_ensemble_step(flbm_ensemble *e, int64_t n)
{
    if (!e) return efail(nullptr, FLBM_E_INVALID, "ensemble is NULL");
    if (n < 0) return efail(e, FLBM_E_INVALID, "n must be >= 0");
    const int rc = launch_steps(e, n);
    if (rc) return rc;
    return check_flags(e);
}

int flbm_ensemble_graph(flbm_ensemble *e, int enable)
{
    if (!e) return efail(nullptr, FLBM_E_INVALID, "ensemble is NULL");
    e->use_graph = enable != 0;
    return FLBM_OK;
}

int flbm_ensemble_set_tuning(flbm_ensemble *e, const flbm_ensemble_tuning *t)
{
    if (!e || !t) return efail(e, FLBM_E_INVALID, "NULL argument");
    const flbm_ensemble_tuning old = e->tune;
    const int rc = apply_tuning(e, *t);
    if (rc != FLBM_OK) {
        const std::string msg = e->err;
        apply_tuning(e, old);
        e->err = msg;
    }
    return rc;
}

int flbm_ensemble_get_tuning(const flbm_ensemble *e, flbm_ensemble_tuning *out)
{
    if (!e || !out) return efail(nullptr, FLBM_E_INVALID, "NULL argument");
    *out = e->tune;
    return FLBM_OK;
}

int flbm_ensemble_autotune(flbm_ensemble *e, int steps_per_trial, flbm_ensemble_tuning *best)
{
    if (!e) return efail(nullptr, FLBM_E_INVALID, "ensemble is NULL");
    if (steps_per_trial < 1) return efail(e, FLBM_E_INVALID, "steps_per_trial must be >= 1");
    if (e->step != 0) return efail(e, FLBM_E_INVALID, "autotune runs only at step 0");
    cudaEvent_t ev[2];
    ECK(e, cudaEventCreate(&ev[0]));
    ECK(e, cudaEventCreate(&ev[1]));
    const bool graph = e->use_graph;
    e->use_graph = false;
    flbm_ensemble_tuning chosen = e->tune;
    double best_ms = 1e300;
    int rc = FLBM_OK;
    const int items[3] = {128, 256, 512}, stages[3] = {2, 3, 4}, warps[2] = {4, 8}, ctas[2] = {1, 2};
    for (int a = 0; a < 3 && rc == FLBM_OK; ++a)
        for (int b = 0; b < 3 && rc == FLBM_OK; ++b)
            for (int w = 0; w < 2 && rc == FLBM_OK; ++w)
                for (int c = 0; c < 2 && rc == FLBM_OK; ++c) {
                    const flbm_ensemble_tuning t{items[a], stages[b], warps[w], ctas[c], 0.0};
                    if (apply_tuning(e, t) != FLBM_OK) continue;   // shape does not fit
                    if (t.ctas_per_sm > 1 && occupancy(e, e->threads, e->smem) < t.ctas_per_sm) continue;
                    rc = launch_steps(e, 2);
                    if (rc) break;
                    if (cudaEventRecord(ev[0], e->stream) != cudaSuccess) { rc = FLBM_E_CUDA; break; }
                    rc = launch_steps(e, steps_per_trial);
                    if (rc) break;
                    if (cudaEventRecord(ev[1], e->stream) != cudaSuccess) { rc = FLBM_E_CUDA; break; }
                    rc = check_flags(e);
                    if (rc) break;
                    float ms = 0.f;
                    if (cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) { rc = FLBM_E_CUDA; break; }
                    const double per = double(ms) / steps_per_trial;
                    if (per < best_ms) {
                        best_ms = per;
                        chosen = t;
                    }
                }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    e->use_graph = graph;
    if (rc == FLBM_E_CUDA && e->err.empty()) e->err = "autotune: CUDA event failure";
    if (rc) return rc;
    rc = apply_tuning(e, chosen);
    if (rc) return rc;
    e->tune.ms_per_step = best_ms < 1e300 ? best_ms : 0.0;
    rc = reset_all(e);
    if (rc) return rc;
    if (best) *best = e->tune;
    return FLBM_OK;
}

int flbm_ensemble_count(const flbm_ensemble *e) { return e ? e->nrep : -1; }

int64_t flbm_ensemble_get_step(const flbm_ensemble *e) { return e ? e->step : -1; }

const char *flbm_ensemble_last_error(const flbm_ensemble *e)
{
    return e ? e->err.c_str() : g_ens_error.c_str();
}

void flbm_ensemble_destroy(flbm_ensemble *e) { release(e); }

}  // extern "C"
