// capi.cu -- the extern "C" boundary declared in include/flbm.h.
//
// Host-side orchestration only: argument checks, device buffers, the AA
// parity bookkeeping, the per-step launch sequence and chunked host<->device
// transfers.  All arithmetic of the method runs in the kernels of
// step_kernel.cuh and aux.cu; S(k) uses cuFFT for the transform.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/flbm.h"
#include "ctx.h"
#include "internal.h"
#include "lattice.cuh"

using namespace flbm;

namespace {

thread_local std::string g_create_error;

constexpr uint64_t kChunkNodes = 1ull << 20;   // nodes per host-transfer chunk

}  // namespace

namespace {

int fail(flbm_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    else g_create_error = msg;
    return code;
}

#define CK(ctx, call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(ctx, FLBM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CKFFT(ctx, call)                                                                  \
    do {                                                                                  \
        cufftResult r_ = (call);                                                          \
        if (r_ != CUFFT_SUCCESS)                                                          \
            return fail(ctx, FLBM_E_CUDA, std::string(#call) + ": cufft error " + std::to_string(int(r_))); \
    } while (0)

size_t elem_size(int prec) { return prec == FLBM_FP64 ? 8 : prec == FLBM_FP32 ? 4 : 2; }

// Slab stride (elements) of the padded population storage of n nodes: slot i
// of node n at i * ns + n, ns = n rounded up to 64 elements plus a pad of
// kSlabPadBytes for slabs of kSlabPadFrom bytes and more, or of FLBM_SLAB_PAD
// bytes (environment, a multiple of 128) at any size when that is set.
// Unpadded, the 27 slabs of a 512^3 FP32 box start 2^29 bytes apart, equal in
// every lower address bit, and the even AA step (which reads and writes the
// same row of all 27 slabs) ran 4.6 % slower than the odd one; a 1 MB pad
// made the step 1.0 % faster (pads of 64 KB to 12 MB: 0.8-1.0 %, 128 B:
// 1.5 % slower).
constexpr uint64_t kSlabPadBytes = uint64_t(1) << 20;
constexpr uint64_t kSlabPadFrom = uint64_t(32) << 20;
uint64_t slab_stride(uint64_t n, size_t es)
{
    uint64_t pad = n * es >= kSlabPadFrom ? kSlabPadBytes : 0;
    if (const char *env = std::getenv("FLBM_SLAB_PAD")) {
        const long long v = std::atoll(env);
        if (v >= 0 && v % 128 == 0 && v <= (1ll << 30)) pad = uint64_t(v);
    }
    return (n + 63) / 64 * 64 + pad / es;
}

int prec_code(const flbm_ctx *c) { return c->p.precision == FLBM_FP64 ? 0 : (c->p.precision == FLBM_FP32 ? 1 : 2); }

int parity(const flbm_ctx *c) { return int((c->step + c->phase) & 1); }

// Whether p is memory the device can address as global memory (device or
// managed); a host pointer handed to a kernel would fault instead of failing.
bool is_device_memory(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // clear the query's error
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

BoxDesc box_of(const flbm_ctx *c)
{
    BoxDesc b;
    b.nx = uint32_t(c->p.nx);
    b.ny = uint32_t(c->p.ny);
    b.nz = uint32_t(c->p.nz);
    b.n = c->n;
    b.ns = c->ns;
    b.rho0 = c->p.rho0;
    b.parity = parity(c);
    return b;
}

}  // namespace

std::string flbm::validate_params(const flbm_params *p)
{
    if (!p) return "params is NULL";
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return "nx, ny, nz must be >= 1";
    const double n = double(p->nx) * double(p->ny) * double(p->nz);
    if (n * 27.0 >= 1099511627776.0) return "box too large (27 N must be < 2^40)";
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return "tau must be finite and > 0.5";
    if (!(p->kT >= 0.0) || !std::isfinite(p->kT)) return "kT must be finite and >= 0";
    if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0)) return "rho0 must be finite and > 0";
    if (p->scheme < FLBM_BGK || p->scheme > FLBM_LEARNED) return "unknown scheme";
    if (p->scheme == FLBM_LEARNED && p->precision != FLBM_FP32)
        return "the learned collision runs on FP32 storage";
    if (p->scheme == FLBM_LEARNED && !(p->kT > 0.0))
        return "the learned collision needs kT > 0 (its feature scale)";
    if (p->precision < FLBM_FP64 || p->precision > FLBM_FP16) return "unknown precision";
    if (p->stats_every < 0) return "stats_every must be >= 0";
    if (p->noise_rho0 != 0 && p->noise_rho0 != 1) return "noise_rho0 must be 0 or 1";
    if (p->noise_stream < 0 || p->noise_stream >= (1 << 24)) return "noise_stream must be in [0, 2^24)";
    if (p->state_form != FLBM_STATE_POPULATIONS && p->state_form != FLBM_STATE_MOMENTS)
        return "unknown state_form";
    if (p->state_form == FLBM_STATE_MOMENTS &&
        (p->precision != FLBM_FP32 || (p->scheme != FLBM_GMF && p->scheme != FLBM_REG)))
        return "the moment-state form runs GMF or Reg on FP32 storage";
    return "";
}

namespace {

// Relaxation and noise scalars of Eq. flbe2 (GMF), Eq. flbe (BGK) and
// Reg-FLBM: post-collision M_k = a_eq,k + lambda_k (m_k - a_eq,k) + phi_k r_k
// with lambda_k = 1 - omega for k = 4..9 (every non-conserved k for BGK),
// phi_k = sqrt(rho kT omega (2 - omega) b_k / c_s^2) (Eq. fluct_phi; all k for
// BGK) and phi_k^g = sqrt(rho kT b_k / c_s^2) for the GMF / Reg ghosts (Eq.
// fluct_phig).  The kernel multiplies amp_h / amp_g by sqrt(rho) and by the
// compile-time sqrt(b_k / c_s^2).
template <typename R>
void mode_coefficients(const flbm_params &p, StepArgs<R> &a)
{
    const double omega = 1.0 / p.tau;
    a.lambda = R(1.0 - omega);
    a.omega = R(omega);
    a.amp_h = R(std::sqrt(p.kT * omega * (2.0 - omega)));
    a.amp_g = p.scheme == FLBM_BGK ? a.amp_h : R(std::sqrt(p.kT));
}

template <typename R>
void fill_constants_t(const flbm_params &p, StepArgs<R> &a)
{
    // Philox4x32-10 key schedule: key = seed, bumped by the Weyl constants
    // (0x9E3779B9, 0xBB67AE85) before each round after the first
    uint32_t k0 = uint32_t(p.seed & 0xffffffffu), k1 = uint32_t(p.seed >> 32);
    for (int r = 0; r < 10; ++r) {
        a.rk[2 * r] = k0;
        a.rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    a.ctr2 = uint32_t(p.noise_stream) << 8;
    // the parts of Philox rounds 0 and 1 that depend only on the launch
    // (counter words 1-3 = step lo, block | ctr2, step hi): round 0 maps word
    // 2 to x0 = hi(M1 c2) ^ step lo ^ k0, y0 = lo(M1 c2); round 1 multiplies
    // x0 by M0 (see philox4x32_10_r2)
    const uint32_t step_lo = uint32_t(a.step), step_hi = uint32_t(a.step >> 32);
    a.ph_zk = step_hi ^ a.rk[1];
    for (int b = 0; b < 6; ++b) {
        const uint64_t p1 = uint64_t(0xCD9E8D57u) * (uint32_t(b) | a.ctr2);
        const uint32_t x0 = uint32_t(p1 >> 32) ^ step_lo ^ a.rk[0];
        const uint64_t q0 = uint64_t(0xD2511F53u) * x0;
        a.ph_u1[b] = uint32_t(p1) ^ a.rk[2];
        a.ph_u2[b] = uint32_t(q0 >> 32) ^ a.rk[3];
        a.ph_u3[b] = uint32_t(q0);
    }
    a.noise_rho0 = p.noise_rho0;
    a.rho0 = R(p.rho0);
    a.sqrt_rho0 = R(std::sqrt(p.rho0));
    mode_coefficients<R>(p, a);
}

template <typename R>
StepArgs<R> make_args(const flbm_ctx *c, int64_t t)
{
    StepArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.nx = uint32_t(c->p.nx);
    a.ny = uint32_t(c->p.ny);
    a.nz = uint32_t(c->p.nz);
    a.cpr = uint32_t((c->p.nx + kBlock - 1) / kBlock);
    a.n = c->n;
    a.ns = c->ns;
    a.nchunks = uint64_t(a.cpr) * a.ny * a.nz;
    a.step = uint64_t(t);
    fill_constants_t<R>(c->p, a);
    a.tx_pad = c->tx_pad;
    a.partials = c->partials;
    a.flag = &c->dflags->flag;
    a.bad_step = &c->dflags->bad_step;
    return a;
}

int reset_flags(flbm_ctx *c)
{
    DevFlags h{0u, 0u, ~0ull};
    CK(c, cudaMemcpyAsync(c->dflags, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    return FLBM_OK;
}

int ensure_pipe(flbm_ctx *c)
{
    if (c->pipe[0]) return FLBM_OK;
    c->pipe_nodes = std::min<uint64_t>(c->n, kChunkNodes);
    for (int b = 0; b < 2; ++b) {
        CK(c, cudaMalloc(&c->pipe[b], c->pipe_nodes * kQ * sizeof(double)));
        CK(c, cudaEventCreateWithFlags(&c->ev_ready[b], cudaEventDisableTiming));
        CK(c, cudaEventCreateWithFlags(&c->ev_free[b], cudaEventDisableTiming));
    }
    CK(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    return FLBM_OK;
}

// Device -> host in chunks of pipe_nodes: produce(buf, n0, cn) fills a
// staging buffer on the context stream, copy(buf, n0, cn) drains it on the
// copy stream; chunk k + 1 is produced while chunk k is copied.
// Moment-state form: rebuild the populations of the current step into the
// population storage (natural AA form) unless they are current already.
int materialise(flbm_ctx *c)
{
    if (c->pops_valid) return FLBM_OK;
    CK(c, launch_ms_export(c->ms[c->ms_cur], static_cast<float *>(c->g), make_args<float>(c, c->step - 1),
                           c->p.scheme, c->ms_grid, c->ms_zseg, c->stream));
    c->phase = int(c->step & 1);
    c->pops_valid = true;
    return FLBM_OK;
}

// The populations were replaced: the next step collides from them.
void populations_written(flbm_ctx *c)
{
    c->ms_live = false;
    c->pops_valid = true;
}

template <typename Produce, typename Copy>
int d2h_chunks(flbm_ctx *c, Produce produce, Copy copy)
{
    int rc = ensure_pipe(c);
    if (rc) return rc;
    int k = 0;
    for (uint64_t n0 = 0; n0 < c->n; n0 += c->pipe_nodes, ++k) {
        const int b = k & 1;
        const uint64_t cn = std::min<uint64_t>(c->pipe_nodes, c->n - n0);
        if (k >= 2) CK(c, cudaStreamWaitEvent(c->stream, c->ev_free[b], 0));
        CK(c, produce(c->pipe[b], n0, cn));
        CK(c, cudaEventRecord(c->ev_ready[b], c->stream));
        CK(c, cudaStreamWaitEvent(c->copy_stream, c->ev_ready[b], 0));
        CK(c, copy(c->pipe[b], n0, cn));
        CK(c, cudaEventRecord(c->ev_free[b], c->copy_stream));
    }
    CK(c, cudaStreamSynchronize(c->copy_stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return FLBM_OK;
}

// Host -> device in chunks: copy(buf, n0, cn) fills a staging buffer on the
// copy stream, consume(buf, n0, cn) scatters it on the context stream.
template <typename Copy, typename Consume>
int h2d_chunks(flbm_ctx *c, Copy copy, Consume consume)
{
    int rc = ensure_pipe(c);
    if (rc) return rc;
    CK(c, cudaEventRecord(c->ev_ready[0], c->stream));   // order after earlier work
    CK(c, cudaStreamWaitEvent(c->copy_stream, c->ev_ready[0], 0));
    int k = 0;
    for (uint64_t n0 = 0; n0 < c->n; n0 += c->pipe_nodes, ++k) {
        const int b = k & 1;
        const uint64_t cn = std::min<uint64_t>(c->pipe_nodes, c->n - n0);
        if (k >= 2) CK(c, cudaStreamWaitEvent(c->copy_stream, c->ev_free[b], 0));
        CK(c, copy(c->pipe[b], n0, cn));
        CK(c, cudaEventRecord(c->ev_ready[b], c->copy_stream));
        CK(c, cudaStreamWaitEvent(c->stream, c->ev_ready[b], 0));
        CK(c, consume(c->pipe[b], n0, cn));
        CK(c, cudaEventRecord(c->ev_free[b], c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return FLBM_OK;
}

}  // namespace

void flbm::destroy_ctx(flbm_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->has_plan) cufftDestroy(c->plan);
    cudaFree(c->fft_in);
    cudaFree(c->fft_out);
    cudaFree(c->shell_s);
    cudaFree(c->shell_c);
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    for (int b = 0; b < 2; ++b) {
        cudaFree(c->pipe[b]);
        if (c->ev_ready[b]) cudaEventDestroy(c->ev_ready[b]);
        if (c->ev_free[b]) cudaEventDestroy(c->ev_free[b]);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    cudaFree(c->partials);
    cudaFree(c->dstats);
    cudaFree(c->dflags);
    if (c->own_g) cudaFree(c->g);
    cudaFree(c->mlp_img);
    cudaFree(c->ms[0]);
    cudaFree(c->ms[1]);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int flbm::create_ctx(const flbm_params *p, void *dev_buf, size_t dev_bytes, void *stream, flbm_ctx **out)
{
    if (!out) return fail(nullptr, FLBM_E_INVALID, "out is NULL");
    *out = nullptr;
    const std::string why = validate_params(p);
    if (!why.empty()) return fail(nullptr, FLBM_E_INVALID, why);
    flbm_ctx *c = new (std::nothrow) flbm_ctx;
    if (!c) return fail(nullptr, FLBM_E_NOMEM, "host allocation failed");
    c->p = *p;
    c->n = uint64_t(p->nx) * uint64_t(p->ny) * uint64_t(p->nz);
    // padded slabs when the buffer holds them: library memory, or a dev_buf
    // of flbm_state_bytes(p); a dev_buf of 27 N elements keeps them unpadded
    c->ns = slab_stride(c->n, elem_size(p->precision));
    if (dev_buf && dev_bytes < c->ns * kQ * elem_size(p->precision)) c->ns = c->n;
    c->g_bytes = c->ns * kQ * elem_size(p->precision);
    int rc = FLBM_OK;
    auto bail = [&](int code) {
        g_create_error = c->err;
        destroy_ctx(c);
        return code;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        c->err = std::string("no usable CUDA device: ") + cudaGetErrorString(e);
        return bail(FLBM_E_CUDA);
    }
    if (stream) {
        c->stream = static_cast<cudaStream_t>(stream);
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return bail(FLBM_E_CUDA); }
        c->own_stream = true;
    }
    if (dev_buf) {
        if (dev_bytes < c->g_bytes) {
            c->err = "dev_buf smaller than flbm_state_bytes()";
            return bail(FLBM_E_NOMEM);
        }
        if (reinterpret_cast<uintptr_t>(dev_buf) % 256 != 0) {
            c->err = "dev_buf must be 256-byte aligned";
            return bail(FLBM_E_INVALID);
        }
        if (!is_device_memory(dev_buf)) {
            c->err = "dev_buf must be device (or managed) memory";
            return bail(FLBM_E_INVALID);
        }
        c->g = dev_buf;
    } else {
        e = cudaMalloc(&c->g, c->g_bytes);
        if (e != cudaSuccess) {
            c->err = std::string("cudaMalloc(populations): ") + cudaGetErrorString(e);
            return bail(FLBM_E_NOMEM);
        }
        c->own_g = true;
    }
    // persistent grids: resident CTAs of the reducing (larger) variants
    int occ = 1, occ_rows = 0;
    if (p->precision == FLBM_FP64)
        step_occupancy_f64(p->scheme, uint32_t(p->nx), true, occ, occ_rows);
    else if (p->precision == FLBM_FP32)
        step_occupancy_f32(p->scheme, uint32_t(p->nx), c->ns, true, occ, occ_rows);
    else
        step_occupancy_f16(p->scheme, uint32_t(p->nx), c->ns, true, occ, occ_rows);
    step_grids(*p, c->nsm, occ, occ_rows, c->grid, c->row_grid);
    // FLBM_INJECT_STARVE=1 (environment, failure-injection tests only): the
    // row pipeline expects 16 bytes more than it copies (the learned step
    // issues no first-layer MMA), so the bounded waits run out and flbm_step
    // reports FLBM_E_TIMEOUT
    if (const char *inj = std::getenv("FLBM_INJECT_STARVE"))
        if (std::atoi(inj) == 1) c->tx_pad = 16;
    if (p->state_form == FLBM_STATE_MOMENTS) {
        for (int b = 0; b < 2; ++b) {
            e = cudaMalloc(&c->ms[b], size_t(kMsVals) * c->n * sizeof(float));
            if (e != cudaSuccess) {
                c->err = std::string("cudaMalloc(moment state): ") + cudaGetErrorString(e);
                return bail(FLBM_E_NOMEM);
            }
        }
        e = ms_prepare(p->scheme, c->nsm, make_args<float>(c, 0), c->ms_grid, c->ms_zseg);
        if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return bail(FLBM_E_CUDA); }
    }
    const int max_grid = std::max(std::max(c->grid, c->row_grid), c->ms_grid);
    e = cudaMalloc(&c->partials, size_t(max_grid) * NSTAT * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->dstats, sizeof(DevStats));
    if (e == cudaSuccess) e = cudaMalloc(&c->dflags, sizeof(DevFlags));
    if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return bail(FLBM_E_NOMEM); }
    e = cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->stream);
    if (e == cudaSuccess) e = launch_fill_rest(c->g, prec_code(c), c->ns * kQ, c->stream);
    if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return bail(FLBM_E_CUDA); }
    rc = reset_flags(c);
    if (rc != FLBM_OK) return bail(rc);
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return bail(FLBM_E_CUDA); }
    *out = c;
    return FLBM_OK;
}

namespace flbm {
void step_grids(const flbm_params &p, int nsm, int occ, int occ_rows, int &grid, int &row_grid)
{
    const uint64_t n = uint64_t(p.nx) * uint64_t(p.ny) * uint64_t(p.nz);
    const uint64_t nchunks = uint64_t((p.nx + kBlock - 1) / kBlock) * p.ny * p.nz;
    // FLBM_CTAS_PER_SM (environment) caps the direct kernel's grid below the
    // occupancy limit; a tuning knob, the default is the occupancy limit
    int per_sm = occ;
    if (const char *env = std::getenv("FLBM_CTAS_PER_SM")) {
        const int v = std::atoi(env);
        if (v > 0 && v < occ) per_sm = v;
    }
    if (p.scheme == FLBM_LEARNED) per_sm = learned_occupancy(n);
    grid = int(std::min<uint64_t>(nchunks, uint64_t(nsm) * per_sm));
    if (grid < 1) grid = 1;
    // FLBM_ROWS=0 (environment) disables the TMA row pipeline
    row_grid = 0;
    const char *rows_env = std::getenv("FLBM_ROWS");
    if (occ_rows > 0 && p.scheme != FLBM_LEARNED && !(rows_env && std::atoi(rows_env) == 0)) {
        const uint64_t nrows = uint64_t(p.ny) * p.nz;
        row_grid = int(std::min<uint64_t>(nrows, uint64_t(nsm) * occ_rows));
    }
}

bool row_pairs_enabled()
{
    const char *e = std::getenv("FLBM_ROW_PAIRS");
    return !(e && std::atoi(e) == 0);
}

void fill_step_constants(const flbm_params &p, StepArgs<float> &a) { fill_constants_t<float>(p, a); }
void fill_step_constants(const flbm_params &p, StepArgs<double> &a) { fill_constants_t<double>(p, a); }
void set_thread_error(const char *msg) { g_create_error = msg; }
}  // namespace flbm

extern "C" {

int flbm_params_init(flbm_params *p, int nx, int ny, int nz, double tau, double kT, double rho0,
                     uint64_t seed, int scheme)
{
    if (!p) return fail(nullptr, FLBM_E_INVALID, "params is NULL");
    std::memset(p, 0, sizeof(*p));
    p->nx = nx;
    p->ny = ny;
    p->nz = nz;
    p->scheme = scheme;
    p->precision = FLBM_FP32;
    p->noise_rho0 = 0;
    p->stats_every = 1;
    p->tau = tau;
    p->kT = kT;
    p->rho0 = rho0;
    p->seed = seed;
    return FLBM_OK;
}

size_t flbm_state_bytes(const flbm_params *p)
{
    if (!validate_params(p).empty()) return 0;
    const size_t es = elem_size(p->precision);
    return slab_stride(uint64_t(p->nx) * uint64_t(p->ny) * uint64_t(p->nz), es) * kQ * es;
}

int flbm_create(int nx, int ny, int nz, double tau, double kT, double rho0, uint64_t seed,
                int scheme, flbm_ctx **out)
{
    flbm_params p;
    flbm_params_init(&p, nx, ny, nz, tau, kT, rho0, seed, scheme);
    return create_ctx(&p, nullptr, 0, nullptr, out);
}

int flbm_create_ex(const flbm_params *p, void *dev_buf, size_t dev_bytes, void *cuda_stream,
                   flbm_ctx **out)
{
    return create_ctx(p, dev_buf, dev_bytes, cuda_stream, out);
}

int flbm_step(flbm_ctx *c, int64_t n)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (c->ens) return fail(c, FLBM_E_INVALID, "an ensemble replica is stepped by flbm_ensemble_step");
    if (n < 0) return fail(c, FLBM_E_INVALID, "n must be >= 0");
    const int every = c->p.stats_every;
    for (int64_t s = 0; s < n; ++s) {
        const int64_t t = c->step + s;
        const bool odd = ((t + c->phase) & 1) != 0;
        const bool stats = every > 0 && (t % every) == 0;
        cudaError_t e;
        if (c->timing) {
            if (c->ev.size() < 2 * (c->ev_used + 1)) {
                for (int k = 0; k < 2; ++k) {
                    cudaEvent_t ev;
                    CK(c, cudaEventCreate(&ev));
                    c->ev.push_back(ev);
                }
            }
            CK(c, cudaEventRecord(c->ev[2 * c->ev_used], c->stream));
        }
        int reduced_grid = c->row_grid > 0 ? c->row_grid : c->grid;   // CTAs that wrote partials
        if (c->p.state_form == FLBM_STATE_MOMENTS) {
            if (!c->ms_live) {   // the first collision, from the populations
                e = launch_ms_boot(static_cast<const float *>(c->g), c->ms[c->ms_cur], make_args<float>(c, t),
                                   c->p.scheme, odd, stats, c->grid, c->stream);
                reduced_grid = c->grid;
                c->ms_live = true;
            } else {
                e = launch_ms_step(c->ms[c->ms_cur], c->ms[c->ms_cur ^ 1], make_args<float>(c, t - 1),
                                   make_args<float>(c, t), c->p.scheme, stats, c->ms_grid, c->ms_zseg,
                                   c->stream);
                reduced_grid = c->ms_grid;
                c->ms_cur ^= 1;
            }
            c->pops_valid = false;
        } else if (c->p.scheme == FLBM_LEARNED) {
            if (!c->mlp_img) return fail(c, FLBM_E_INVALID, "set the network (flbm_set_mlp) before stepping");
            const double w[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
            LearnArgs L;
            L.img = c->mlp_img;
            for (int k = 0; k < 4; ++k) L.inv_s[k] = float(1.0 / std::sqrt(c->p.rho0 * c->p.kT * w[k] * 3.0));
            L.sig3 = float(std::pow(c->p.kT / c->p.rho0, 1.5));
            L.x27 = float(1.0 / c->p.tau - 1.0);
            L.starve = c->tx_pad != 0;   // FLBM_INJECT_STARVE=1 (tests)
            e = launch_step_learned(static_cast<float *>(c->g), make_args<float>(c, t), L, odd, stats, c->grid,
                                    c->stream);
        } else if (c->p.precision == FLBM_FP64)
            e = launch_step_f64(static_cast<double *>(c->g), make_args<double>(c, t), c->p.scheme, odd,
                                stats, c->grid, c->row_grid, c->stream);
        else if (c->p.precision == FLBM_FP32)
            e = launch_step_f32(static_cast<float *>(c->g), make_args<float>(c, t), c->p.scheme, odd,
                                stats, c->grid, c->row_grid, c->stream);
        else
            e = launch_step_f16(c->g, make_args<float>(c, t), c->p.scheme, odd, stats, c->grid,
                                c->row_grid, c->stream);
        if (e != cudaSuccess) return fail(c, FLBM_E_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
        if (c->timing) {
            CK(c, cudaEventRecord(c->ev[2 * c->ev_used + 1], c->stream));
            ++c->ev_used;
        }
        if (stats) {
            e = launch_stats_finalize(c->partials, reduced_grid, c->dstats, t, double(c->n), c->stream);
            if (e != cudaSuccess) return fail(c, FLBM_E_CUDA, std::string("stats launch: ") + cudaGetErrorString(e));
        }
    }
    c->step += n;
    DevFlags h;
    CK(c, cudaMemcpyAsync(&h, c->dflags, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (h.flag & 2u)
        return fail(c, FLBM_E_TIMEOUT, "a bounded device wait ran out during the last steps");
    if (h.flag) {
        c->step = int64_t(h.bad_step);
        return fail(c, FLBM_E_UNSTABLE, "instability: rho <= 0 or non-finite at step " +
                                            std::to_string(int64_t(h.bad_step)));
    }
    return FLBM_OK;
}

int flbm_moments(flbm_ctx *c, double *rho, double *j, double *pi)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (int rc = materialise(c)) return rc;
    const BoxDesc b = box_of(c);
    const uint64_t N = c->n;
    const int prec = prec_code(c);
    return d2h_chunks(
        c, [&](double *buf, uint64_t n0, uint64_t cn) { return launch_moments(c->g, prec, b, n0, cn, buf, c->stream); },
        [&](double *buf, uint64_t n0, uint64_t cn) {
            const size_t w = cn * sizeof(double);
            cudaError_t e = cudaSuccess;
            if (rho) e = cudaMemcpyAsync(rho + n0, buf, w, cudaMemcpyDeviceToHost, c->copy_stream);
            if (e == cudaSuccess && j)
                e = cudaMemcpy2DAsync(j + n0, N * sizeof(double), buf + cn, w, w, 3, cudaMemcpyDeviceToHost,
                                      c->copy_stream);
            if (e == cudaSuccess && pi)
                e = cudaMemcpy2DAsync(pi + n0, N * sizeof(double), buf + 4 * cn, w, w, 6,
                                      cudaMemcpyDeviceToHost, c->copy_stream);
            return e;
        });
}

int flbm_stats(flbm_ctx *c, flbm_stats_t *out)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (!out) return fail(c, FLBM_E_INVALID, "out is NULL");
    DevStats h;
    CK(c, cudaMemcpyAsync(&h, c->dstats, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    std::memset(out, 0, sizeof(*out));
    const double N = double(c->n);
    out->step = h.nsamp ? h.step : -1;
    out->n_samples = h.nsamp;
    out->mass = N * c->p.rho0 + h.last[S_DRHO];
    for (int a = 0; a < 3; ++a) {
        out->mom[a] = h.last[S_JX + a];
        out->u2[a] = h.last[S_UX2 + a] / N;
        out->u2_avg[a] = h.nsamp ? h.acc_u2[a] / double(h.nsamp) : 0.0;
    }
    const double th[4] = {3.0, 3.0, 5.0, 1.0};
    for (int k = 0; k < 4; ++k) {
        if (!h.nsamp) continue;
        const double m = h.acc_m[k] / double(h.nsamp);
        const double m2 = h.acc_m2[k] / double(h.nsamp);
        out->m_mean[k] = m;
        out->m_var[k] = m2 - m * m;
        const double t = th[k] * c->p.rho0 * c->p.kT;
        out->er[k] = t > 0 ? out->m_var[k] / t : 0.0;
    }
    return FLBM_OK;
}

int flbm_stats_reset(flbm_ctx *c)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    CK(c, cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return FLBM_OK;
}

int flbm_structure_factor(flbm_ctx *c, int observable, int nshell, double *S, int64_t *count)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (observable < FLBM_OBS_RHO || observable > FLBM_OBS_JZ) return fail(c, FLBM_E_INVALID, "unknown observable");
    if (nshell < 1 || nshell > 3072) return fail(c, FLBM_E_INVALID, "nshell must be in [1, 3072]");
    if (!S || !count) return fail(c, FLBM_E_INVALID, "S and count must not be NULL");
    if (int rc = materialise(c)) return rc;
    const bool dbl = c->p.precision == FLBM_FP64;
    const size_t rs = dbl ? sizeof(double) : sizeof(float);
    const uint64_t nspec = uint64_t(c->p.nx / 2 + 1) * c->p.ny * c->p.nz;
    if (!c->has_plan) {
        CK(c, cudaMalloc(&c->fft_in, c->n * rs));
        CK(c, cudaMalloc(&c->fft_out, nspec * 2 * rs));
        CKFFT(c, cufftPlan3d(&c->plan, c->p.nz, c->p.ny, c->p.nx, dbl ? CUFFT_D2Z : CUFFT_R2C));
        c->has_plan = true;
    }
    CKFFT(c, cufftSetStream(c->plan, c->stream));
    if (nshell > c->shell_cap) {
        cudaFree(c->shell_s);
        cudaFree(c->shell_c);
        c->shell_s = nullptr;
        c->shell_c = nullptr;
        c->shell_cap = 0;
        CK(c, cudaMalloc(&c->shell_s, nshell * sizeof(double)));
        CK(c, cudaMalloc(&c->shell_c, nshell * sizeof(unsigned long long)));
        c->shell_cap = nshell;
    }
    const BoxDesc b = box_of(c);
    CK(c, launch_observable(c->g, prec_code(c), b, observable, c->fft_in, c->stream));
    if (dbl)
        CKFFT(c, cufftExecD2Z(c->plan, static_cast<cufftDoubleReal *>(c->fft_in),
                              static_cast<cufftDoubleComplex *>(c->fft_out)));
    else
        CKFFT(c, cufftExecR2C(c->plan, static_cast<cufftReal *>(c->fft_in),
                              static_cast<cufftComplex *>(c->fft_out)));
    CK(c, cudaMemsetAsync(c->shell_s, 0, nshell * sizeof(double), c->stream));
    CK(c, cudaMemsetAsync(c->shell_c, 0, nshell * sizeof(unsigned long long), c->stream));
    CK(c, launch_shells(c->fft_out, prec_code(c), b, nshell, c->shell_s, c->shell_c, c->stream));
    CK(c, cudaMemcpyAsync(S, c->shell_s, nshell * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(count, c->shell_c, nshell * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    for (int s = 0; s < nshell; ++s)
        if (count[s] > 0) S[s] /= double(count[s]);
    return FLBM_OK;
}

int flbm_spectral_er(flbm_ctx *c, int observable, int nshell, double *er, int64_t *count)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (!(c->p.kT > 0.0)) return fail(c, FLBM_E_INVALID, "the spectral ER needs kT > 0");
    const int rc = flbm_structure_factor(c, observable, nshell, er, count);
    if (rc != FLBM_OK) return rc;
    // flat S_m^th of the lattice invariant measure <dg_i dg_j> = (rho0 kT /
    // c_s^2) w_i delta_ij, per node
    static const double factor[7] = {3.0, 3.0, 5.0, 1.0, 1.0, 1.0, 1.0};
    const double th = factor[observable] * c->p.rho0 * c->p.kT;
    for (int s = 0; s < nshell; ++s) er[s] = count[s] > 0 ? er[s] / th : 0.0;
    return FLBM_OK;
}

int flbm_get_populations(flbm_ctx *c, double *f)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (!f) return fail(c, FLBM_E_INVALID, "f is NULL");
    if (int rc = materialise(c)) return rc;
    const BoxDesc b = box_of(c);
    const uint64_t N = c->n;
    const int prec = prec_code(c);
    return d2h_chunks(
        c, [&](double *buf, uint64_t n0, uint64_t cn) {
            return launch_gather_f(c->g, prec, b, n0, cn, buf, false, c->stream);
        },
        [&](double *buf, uint64_t n0, uint64_t cn) {
            const size_t w = cn * sizeof(double);
            return cudaMemcpy2DAsync(f + n0, N * sizeof(double), buf, w, w, kQ, cudaMemcpyDeviceToHost,
                                     c->copy_stream);
        });
}

}  // extern "C"

namespace {

// An ensemble replica's state may be replaced only while the ensemble's
// storage is in the natural form (every replica shares the AA parity).
int replica_state_check(flbm_ctx *c)
{
    if (c->ens && parity(c) != 0)
        return fail(c, FLBM_E_INVALID,
                    "an ensemble replica's state can be replaced only when its storage is in the "
                    "natural form (an even number of ensemble steps since the last replacement)");
    return FLBM_OK;
}

int state_replaced(flbm_ctx *c)
{
    if (c->ens) ensemble_state_replaced(c->ens);
    return FLBM_OK;
}

}  // namespace

extern "C" {

int flbm_set_populations(flbm_ctx *c, const double *f)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (!f) return fail(c, FLBM_E_INVALID, "f is NULL");
    if (int rc = replica_state_check(c)) return rc;
    BoxDesc b = box_of(c);
    b.parity = 0;
    const uint64_t N = c->n;
    const int prec = prec_code(c);
    int rc = h2d_chunks(
        c, [&](double *buf, uint64_t n0, uint64_t cn) {
            const size_t w = cn * sizeof(double);
            return cudaMemcpy2DAsync(buf, w, f + n0, N * sizeof(double), w, kQ, cudaMemcpyHostToDevice,
                                     c->copy_stream);
        },
        [&](double *buf, uint64_t n0, uint64_t cn) {
            return launch_scatter_f(c->g, prec, b, n0, cn, buf, c->stream);
        });
    if (rc) return rc;
    c->phase = int(c->step & 1);   // natural form at the current step
    populations_written(c);
    rc = reset_flags(c);
    if (rc) return rc;
    CK(c, cudaStreamSynchronize(c->stream));
    return state_replaced(c);
}

int flbm_init_thermal(flbm_ctx *c, uint64_t seed)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (int rc = replica_state_check(c)) return rc;
    BoxDesc b = box_of(c);
    b.parity = 0;
    CK(c, launch_init_thermal(c->g, prec_code(c), b, c->p.kT, seed, c->stream));
    c->phase = int(c->step & 1);   // natural form at the current step
    populations_written(c);
    int rc = reset_flags(c);
    if (rc) return rc;
    CK(c, cudaStreamSynchronize(c->stream));
    return state_replaced(c);
}

int flbm_probe(flbm_ctx *c, const int64_t *nodes, int64_t count, double *f)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (count < 0 || (count > 0 && (!nodes || !f))) return fail(c, FLBM_E_INVALID, "bad probe arguments");
    for (int64_t k = 0; k < count; ++k)
        if (nodes[k] < 0 || uint64_t(nodes[k]) >= c->n)
            return fail(c, FLBM_E_INVALID, "probe node index out of range");
    if (int rc = materialise(c)) return rc;
    int rc = ensure_pipe(c);
    if (rc) return rc;
    const BoxDesc b = box_of(c);
    // a staging buffer holds pipe_nodes * 27 doubles: node list + 27 outputs per node
    const int64_t chunk = int64_t(c->pipe_nodes * kQ / (kQ + 1));
    long long *dn = reinterpret_cast<long long *>(c->pipe[0]);
    for (int64_t k0 = 0; k0 < count; k0 += chunk) {
        const int64_t cn = std::min<int64_t>(chunk, count - k0);
        double *dout = c->pipe[0] + chunk;
        CK(c, cudaMemcpyAsync(dn, nodes + k0, cn * sizeof(long long), cudaMemcpyHostToDevice, c->stream));
        CK(c, launch_probe(c->g, prec_code(c), b, dn, cn, dout, c->stream));
        CK(c, cudaMemcpyAsync(f + k0 * kQ, dout, cn * kQ * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return FLBM_OK;
}

int flbm_get_state(flbm_ctx *c, void *host)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (!host) return fail(c, FLBM_E_INVALID, "host is NULL");
    if (int rc = materialise(c)) return rc;
    const size_t es = elem_size(c->p.precision);
    if (parity(c) == 0) {
        // natural form: the host layout is the 27 slabs without their pads
        const size_t slab = c->n * es;
        if (c->ns == c->n) {
            CK(c, cudaMemcpyAsync(host, c->g, kQ * slab, cudaMemcpyDeviceToHost, c->stream));
        } else {
            for (int i = 0; i < kQ; ++i)
                CK(c, cudaMemcpyAsync(static_cast<char *>(host) + i * slab,
                                      static_cast<const char *>(c->g) + i * c->ns * es, slab,
                                      cudaMemcpyDeviceToHost, c->stream));
        }
    } else {
        const BoxDesc b = box_of(c);
        const uint64_t N = c->n;
        const int prec = prec_code(c);
        return d2h_chunks(
            c, [&](double *buf, uint64_t n0, uint64_t cn) {
                return launch_gather_state(c->g, prec, b, n0, cn, buf, c->stream);
            },
            [&](double *buf, uint64_t n0, uint64_t cn) {
                return cudaMemcpy2DAsync(static_cast<char *>(host) + n0 * es, N * es, buf, cn * es, cn * es,
                                         kQ, cudaMemcpyDeviceToHost, c->copy_stream);
            });
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return FLBM_OK;
}

int flbm_set_state(flbm_ctx *c, const void *host)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (!host) return fail(c, FLBM_E_INVALID, "host is NULL");
    if (int rc = replica_state_check(c)) return rc;
    const size_t es = elem_size(c->p.precision), slab = c->n * es;
    if (c->ns == c->n) {
        CK(c, cudaMemcpyAsync(c->g, host, kQ * slab, cudaMemcpyHostToDevice, c->stream));
    } else {
        for (int i = 0; i < kQ; ++i)
            CK(c, cudaMemcpyAsync(static_cast<char *>(c->g) + i * c->ns * es,
                                  static_cast<const char *>(host) + i * slab, slab, cudaMemcpyHostToDevice,
                                  c->stream));
    }
    c->phase = int(c->step & 1);
    populations_written(c);
    int rc = reset_flags(c);
    if (rc) return rc;
    CK(c, cudaStreamSynchronize(c->stream));
    return state_replaced(c);
}

int flbm_set_mlp(flbm_ctx *c, const float *params)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (!params) return fail(c, FLBM_E_INVALID, "params is NULL");
    if (c->p.scheme != FLBM_LEARNED) return fail(c, FLBM_E_INVALID, "the context's scheme is not FLBM_LEARNED");
    std::vector<unsigned char> img;
    build_mlp_image(params, img);
    if (!c->mlp_img) CK(c, cudaMalloc(&c->mlp_img, img.size()));
    CK(c, cudaMemcpyAsync(c->mlp_img, img.data(), img.size(), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return FLBM_OK;
}

int flbm_mlp_pairs(flbm_ctx *c, float *dev_x, float *dev_t)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (!dev_x || !dev_t) return fail(c, FLBM_E_INVALID, "dev_x and dev_t must not be NULL");
    if (!is_device_memory(dev_x) || !is_device_memory(dev_t))
        return fail(c, FLBM_E_INVALID, "dev_x and dev_t must be device (or managed) memory");
    if (!(c->p.kT > 0.0)) return fail(c, FLBM_E_INVALID, "training pairs need kT > 0 (the feature scale)");
    if (int rc = materialise(c)) return rc;
    int rc = ensure_pipe(c);
    if (rc) return rc;
    const BoxDesc b = box_of(c);
    const int prec = prec_code(c);
    for (uint64_t n0 = 0; n0 < c->n; n0 += c->pipe_nodes) {
        const uint64_t cn = std::min<uint64_t>(c->pipe_nodes, c->n - n0);
        CK(c, launch_gather_f(c->g, prec, b, n0, cn, c->pipe[0], true, c->stream));
        CK(c, launch_mlp_pairs(c->pipe[0], cn, c->p.rho0, c->p.kT, 1.0 / c->p.tau, dev_x + n0 * 28,
                               dev_t + n0 * 27, c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return FLBM_OK;
}

int flbm_timing_enable(flbm_ctx *c, int enable)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    c->timing = enable != 0;
    c->ev_used = 0;
    return FLBM_OK;
}

int flbm_timing_read(flbm_ctx *c, double *kernel_ms, int64_t *launches)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (!kernel_ms || !launches) return fail(c, FLBM_E_INVALID, "NULL output");
    double tot = 0.0;
    for (size_t k = 0; k < c->ev_used; ++k) {
        CK(c, cudaEventSynchronize(c->ev[2 * k + 1]));
        float ms = 0.f;
        CK(c, cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]));
        tot += ms;
    }
    *kernel_ms = tot;
    *launches = int64_t(c->ev_used);
    c->ev_used = 0;
    return FLBM_OK;
}

int64_t flbm_get_step(const flbm_ctx *c) { return c ? c->step : -1; }

int flbm_set_step(flbm_ctx *c, int64_t step)
{
    if (!c) return fail(nullptr, FLBM_E_INVALID, "ctx is NULL");
    if (step < 0) return fail(c, FLBM_E_INVALID, "step must be >= 0");
    if (c->ens) return fail(c, FLBM_E_INVALID, "an ensemble replica follows the ensemble's step");
    // the moment state's noise is keyed on the step it was made at: continue
    // from the populations
    if (int rc = materialise(c)) return rc;
    populations_written(c);
    const int par = parity(c);
    c->step = step;
    c->phase = int((par - (step & 1)) & 1);
    return FLBM_OK;
}

int flbm_get_params(const flbm_ctx *c, flbm_params *out)
{
    if (!c || !out) return fail(nullptr, FLBM_E_INVALID, "NULL argument");
    *out = c->p;
    return FLBM_OK;
}

const char *flbm_last_error(const flbm_ctx *c)
{
    return c ? c->err.c_str() : g_create_error.c_str();
}

void flbm_destroy(flbm_ctx *c)
{
    if (c && c->ens) return;   // a replica lives and dies with its ensemble
    destroy_ctx(c);
}

}  // extern "C"
