// flb_api.cu -- the C ABI declared in include/flb.h: context object, buffer
// management, step sequencing, observables, checkpoints and error reporting.
// All compute happens in the kernels of flb_prec.cuh / flb_fft.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/flb.h"
#include "flb_internal.h"

using flb::HostModel;
using flb::PrecOps;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

}  // namespace

namespace flb {
int set_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace flb

namespace {

#define FLB_CUDA(call)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(e_ == cudaErrorMemoryAllocation ? FLB_ENOMEM : FLB_ECUDA,                   \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

// Makes the context's device current for the duration of an API call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (dev >= 0 && dev != prev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

constexpr char kMagic[8] = {'F', 'L', 'B', 'C', 'K', 'P', 'T', '1'};

}  // namespace

struct flb_ctx {
    HostModel m{};
    flb_free_energy fe{};
    int prec = FLB_FP32;
    int device = 0;
    cudaStream_t stream = nullptr;
    int check_every = 0;
    // guard zones (opt.guard): allocation base of each guarded buffer; the
    // buffer itself starts kGuardBytes after it
    struct GuardZone {
        void* base;
        size_t bytes;
        const char* name;
    };
    std::vector<GuardZone> guards;
    int guard = 0;
    // z-chunk autotuning of the z-marching step (opt.z_chunk = 0): candidate
    // lengths, the best time of each, CUDA events of the tuning launches
    struct ZTune {
        bool active = false;
        std::vector<int> cand;
        std::vector<float> best;
        std::vector<cudaEvent_t> ev;
        int issued = 0;
    } zt;
    const PrecOps* ops = nullptr;
    uint64_t step = 0;

    void* buf[2] = {nullptr, nullptr};  // post-collision populations of the last step
    int cur = 0;
    void* drho = nullptr;               // density deviation field (compute type)
    void* mu = nullptr;                 // chemical potential (observables)
    void* F = nullptr;                  // force field, 3 components (observables)
    double* partials = nullptr;         // per-block reduction rows
    double* red = nullptr;              // reduced columns (device)
    double2* fft = nullptr;             // FFT work array
    double2* fft_scratch = nullptr;
    double* sk_tmp = nullptr;
    std::vector<double*> sk_acc;        // per-mode structure factor accumulators
    std::vector<int> sk_count;
    std::vector<double> mv_sum;         // per-mode sum over snapshots of the site variance
    int mv_count = 0;

    // modified-equilibrium model: Cholesky table and the two noise fields
    double* sw_chol = nullptr;
    double2* sw_work = nullptr;
    double2* sw_xi = nullptr;

    // interface heights and height spectrum of a stripe
    double* h_dev = nullptr;            // 2 X heights
    double2* hs_work = nullptr;         // 2 X complex
    double2* hs_scratch = nullptr;
    double* hs_acc = nullptr;           // X
    double* hs_tmp = nullptr;
    int hs_count = 0;

    // adjoint scratch
    void* adj_work = nullptr;
    double* adj_rows = nullptr;
    void* adj_lam2 = nullptr;  // flb_adjoint_segment: second adjoint state (ping-pong)
    void* adj_rb = nullptr;    // flb_adjoint_segment: deferred density parts (2 fields)
    double* ss_dev = nullptr;  // flb_step_sums: 4 sums per step (device)
    size_t ss_cap = 0;

    // kernel timing
    bool timing = false;
    double t_ms[FLB_NKERNEL_TIMERS] = {0, 0, 0};
    int t_n[FLB_NKERNEL_TIMERS] = {0, 0, 0};
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_pending;  // (kernel id, index of start event)
    size_t ev_used = 0;

    size_t pop_bytes() const { return (size_t)m.Q * m.V * ops->elem_size; }
    size_t field_bytes() const { return (size_t)m.V * ops->real_size; }
};

namespace {

int alloc(void** p, size_t bytes)
{
    if (*p) return FLB_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? FLB_ENOMEM : FLB_ECUDA,
                    std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    return FLB_OK;
}

constexpr size_t kGuardBytes = 65536;
constexpr unsigned char kGuardByte = 0xA5;

// alloc() with guard zones on both sides when the context asks for them.
int alloc_guarded(flb_ctx* c, void** p, size_t bytes, const char* name)
{
    if (!c->guard) return alloc(p, bytes);
    if (*p) return FLB_OK;
    void* base = nullptr;
    int rc = alloc(&base, bytes + 2 * kGuardBytes);
    if (rc) return rc;
    char* user = (char*)base + kGuardBytes;
    cudaError_t e = cudaMemsetAsync(base, kGuardByte, kGuardBytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(user + bytes, kGuardByte, kGuardBytes, c->stream);
    if (e != cudaSuccess) {
        cudaFree(base);
        return fail(FLB_ECUDA, std::string("guard zones: ") + cudaGetErrorString(e));
    }
    c->guards.push_back({base, bytes, name});
    *p = user;
    return FLB_OK;
}

void free_all(flb_ctx* c)
{
    void* ptrs[] = {c->buf[0], c->buf[1], c->drho, c->mu, c->F, c->partials, c->red, c->fft, c->fft_scratch, c->sk_tmp,
                    c->adj_work, c->adj_rows, c->adj_lam2, c->adj_rb, c->ss_dev, c->h_dev, c->hs_work, c->hs_scratch, c->hs_acc,
                    c->hs_tmp, c->sw_chol, c->sw_work, c->sw_xi};
    for (void* p : ptrs) {
        bool guarded = false;
        for (const auto& g : c->guards) guarded |= p == (char*)g.base + kGuardBytes;
        if (p && !guarded) cudaFree(p);
    }
    for (const auto& g : c->guards) cudaFree(g.base);
    c->guards.clear();
    for (cudaEvent_t e : c->zt.ev) cudaEventDestroy(e);
    c->zt.ev.clear();
    for (double* p : c->sk_acc)
        if (p) cudaFree(p);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
}

// Timing: start/stop events around one kernel launch.
int timer_begin(flb_ctx* c, int id, size_t* slot)
{
    if (!c->timing) return FLB_OK;
    while (c->ev_pool.size() < c->ev_used + 2) {
        cudaEvent_t e;
        FLB_CUDA(cudaEventCreate(&e));
        c->ev_pool.push_back(e);
    }
    *slot = c->ev_used;
    c->ev_used += 2;
    c->ev_pending.push_back({id, (int)*slot});
    FLB_CUDA(cudaEventRecord(c->ev_pool[*slot], c->stream));
    return FLB_OK;
}
int timer_end(flb_ctx* c, size_t slot)
{
    if (!c->timing) return FLB_OK;
    FLB_CUDA(cudaEventRecord(c->ev_pool[slot + 1], c->stream));
    return FLB_OK;
}
int timer_flush(flb_ctx* c)
{
    if (c->ev_pending.empty()) return FLB_OK;
    FLB_CUDA(cudaStreamSynchronize(c->stream));
    for (auto& pe : c->ev_pending) {
        float ms = 0.f;
        FLB_CUDA(cudaEventElapsedTime(&ms, c->ev_pool[pe.second], c->ev_pool[pe.second + 1]));
        c->t_ms[pe.first] += ms;
        c->t_n[pe.first] += 1;
    }
    c->ev_pending.clear();
    c->ev_used = 0;
    return FLB_OK;
}

const PrecOps* ops_for(int prec)
{
    switch (prec) {
    case FLB_FP64: return &flb::ops_fp64();
    case FLB_FP32: return &flb::ops_fp32();
    case FLB_BF16: return &flb::ops_bf16();
    default: return nullptr;
    }
}

int ensure_partials(flb_ctx* c)
{
    int rc = alloc((void**)&c->partials, (size_t)c->ops->partial_rows_max(c->m) * 2 * c->m.Q * sizeof(double));
    if (rc) return rc;
    return alloc((void**)&c->red, 64 * sizeof(double));
}

// Reduce per-block partial rows into ncol doubles on the host.
int reduce_to_host(flb_ctx* c, int nrows, int ncol, double* host)
{
    FLB_CUDA(flb::sum_columns(c->partials, nrows, ncol, c->red, c->stream));
    FLB_CUDA(cudaMemcpyAsync(host, c->red, ncol * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    FLB_CUDA(cudaStreamSynchronize(c->stream));
    return FLB_OK;
}

// z-chunk autotuning of the z-marching step (D3Q19 non-ideal, opt.z_chunk = 0).
// Candidates: for every block count nc from ceil(Z/40) to ceil(Z/12) the
// balanced length ceil(Z/nc), at most 16 of them; each is launched
// kZTuneRounds times (the candidates in turn) with CUDA events around it and
// the fastest launch decides.  The steps are the
// caller's own steps: the chunk length changes no result.
constexpr int kZTuneRounds = 3;

void ztune_start(flb_ctx* c)
{
    const HostModel& m = c->m;
    if (m.zchunk != 0 || m.Q != 19 || !m.nonideal || m.Z <= 16) return;
    std::vector<int> all;
    for (int nc = (m.Z + 39) / 40; nc <= (m.Z + 11) / 12; ++nc) {
        const int len = (m.Z + nc - 1) / nc;
        if (all.empty() || all.back() != len) all.push_back(len);
    }
    std::vector<int> cand;
    const size_t n = std::min<size_t>(all.size(), 16);
    for (size_t k = 0; k < n; ++k) cand.push_back(all[k * all.size() / n]);
    if (cand.size() < 2) return;
    std::vector<cudaEvent_t> ev(2 * kZTuneRounds * cand.size());
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            for (auto& f : ev)
                if (f) cudaEventDestroy(f);
            return;  // no tuning: the built-in default length
        }
    c->zt.cand = cand;
    c->zt.best.assign(cand.size(), 3.0e38f);
    c->zt.ev = ev;
    c->zt.issued = 0;
    c->zt.active = true;
}

// All tuning launches issued: wait for them, keep the fastest length.
int ztune_finish(flb_ctx* c)
{
    auto& z = c->zt;
    for (int k = 0; k < z.issued; ++k) {
        float ms = 0.f;
        // the launches may span a flb_set_stream: wait on each launch's own event
        FLB_CUDA(cudaEventSynchronize(z.ev[2 * k + 1]));
        FLB_CUDA(cudaEventElapsedTime(&ms, z.ev[2 * k], z.ev[2 * k + 1]));
        float& b = z.best[k % z.cand.size()];
        b = std::min(b, ms);
    }
    const size_t i = std::min_element(z.best.begin(), z.best.end()) - z.best.begin();
    c->m.zchunk = z.cand[i];
    for (cudaEvent_t e : z.ev) cudaEventDestroy(e);
    z.ev.clear();
    z.active = false;
    return FLB_OK;
}

int conservation(flb_ctx* c, double out[4])
{
    int rc = ensure_partials(c);
    if (rc) return rc;
    int nrows = 0;
    FLB_CUDA(c->ops->cons_partials(c->m, c->buf[c->cur], c->partials, &nrows, c->stream));
    double h[4];
    rc = reduce_to_host(c, nrows, 4, h);
    if (rc) return rc;
    out[0] = c->m.rho0 * (double)c->m.V + h[0];
    out[1] = h[1];
    out[2] = h[2];
    out[3] = h[3];
    return FLB_OK;
}

int validate(int lattice, const int dims[3], double om_s, double om_b, double om_g, double kT,
             const flb_free_energy* fe, const flb_options& o)
{
    if (lattice != FLB_D2Q9 && lattice != FLB_D3Q19) return fail(FLB_EINVAL, "lattice must be FLB_D2Q9 or FLB_D3Q19");
    if (!dims) return fail(FLB_EINVAL, "dims is NULL");
    for (int d = 0; d < 3; ++d)
        if (dims[d] < 1) return fail(FLB_EINVAL, "every dimension must be >= 1");
    if (lattice == FLB_D2Q9 && dims[2] != 1) return fail(FLB_EINVAL, "D2Q9 needs dims[2] == 1");
    const double V = (double)dims[0] * dims[1] * dims[2];
    if (V >= 2147483648.0) return fail(FLB_EINVAL, "X*Y*Z must be below 2^31");
    if (dims[1] > 65535 * 8 || dims[2] > 65535 * 4) return fail(FLB_EINVAL, "Y or Z too large for the launch grid");
    const double oms[3] = {om_s, om_b, om_g};
    for (double om : oms)
        if (!(om > 0.0 && om < 2.0)) return fail(FLB_EINVAL, "relaxation rates must lie in (0, 2)");
    if (!(o.rho0 > 0.0) || !std::isfinite(o.rho0)) return fail(FLB_EINVAL, "rho0 must be positive");
    // Sec. VI: |u| << cs together with <j j> = rho0 kT bounds kT by cs^2 rho0
    if (!(kT >= 0.0) || !(kT <= o.rho0 / 3.0)) return fail(FLB_EINVAL, "kT must lie in [0, cs^2 rho0]");
    if (o.precision != FLB_FP64 && o.precision != FLB_FP32 && o.precision != FLB_BF16)
        return fail(FLB_EINVAL, "unknown precision");
    if (o.check_every < 0) return fail(FLB_EINVAL, "check_every must be >= 0");
    if (o.guard != 0 && o.guard != 1) return fail(FLB_EINVAL, "guard must be 0 or 1");
    if (o.z_chunk < 0) return fail(FLB_EINVAL, "z_chunk must be >= 0");
    if (o.z_chunk > 0 && (dims[2] + o.z_chunk - 1) / o.z_chunk > 65535)
        return fail(FLB_EINVAL, "z_chunk too small for the launch grid (Z / z_chunk must be <= 65535)");
    if (fe && fe->enabled) {
        const double v[4] = {fe->A, fe->B, fe->rho_c, fe->kappa};
        for (double x : v)
            if (!std::isfinite(x)) return fail(FLB_EINVAL, "free-energy parameters must be finite");
        if (fe->kappa < 0.0) return fail(FLB_EINVAL, "kappa must be >= 0");
        if (fe->model != 0 && fe->model != 1) return fail(FLB_EINVAL, "free-energy model must be 0 or 1");
        if (fe->model == 1 && lattice != FLB_D2Q9)
            return fail(FLB_EINVAL, "the modified-equilibrium model is defined for D2Q9 only");
    }
    return FLB_OK;
}

}  // namespace

extern "C" {

void flb_default_options(flb_options* o)
{
    if (!o) return;
    o->precision = FLB_FP32;
    o->rho0 = 1.0;
    o->replica = 0;
    o->noise_rho_local = 1;
    o->stream = nullptr;
    o->device = -1;
    o->check_every = 0;
    o->guard = 0;
    o->z_chunk = 0;
}

int flb_create(flb_ctx** out, int lattice, const int dims[3], double omega_shear, double omega_bulk,
               double omega_ghost, double kT, const flb_free_energy* fe, uint64_t seed, const flb_options* opt)
{
    FLB_TRACE();
    if (!out) return fail(FLB_EINVAL, "out is NULL");
    *out = nullptr;
    flb_options o;
    flb_default_options(&o);
    if (opt) o = *opt;
    int rc = validate(lattice, dims, omega_shear, omega_bulk, omega_ghost, kT, fe, o);
    if (rc) return rc;

    flb_ctx* c = new (std::nothrow) flb_ctx();
    if (!c) return fail(FLB_ENOMEM, "host allocation failed");
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        delete c;
        return fail(FLB_ECUDA, "no CUDA device");
    }
    DeviceGuard guard(dev);
    if (!guard.ok) {
        delete c;
        return fail(FLB_ECUDA, "cudaSetDevice failed");
    }
    c->device = dev;
    c->prec = o.precision;
    c->ops = ops_for(o.precision);
    c->stream = (cudaStream_t)o.stream;
    c->check_every = o.check_every;
    c->guard = o.guard;
    HostModel& m = c->m;
    m.zchunk = o.z_chunk;
    m.Q = lattice;
    m.D = lattice == FLB_D2Q9 ? 2 : 3;
    m.X = dims[0];
    m.Y = dims[1];
    m.Z = dims[2];
    m.V = (long)dims[0] * dims[1] * dims[2];
    m.rho0 = o.rho0;
    m.om_s = omega_shear;
    m.om_b = omega_bulk;
    m.om_g = omega_ghost;
    m.kT = kT;
    m.seed = seed;
    m.replica = o.replica;
    m.noise_local = o.noise_rho_local ? 1 : 0;
    if (fe && fe->enabled) {
        c->fe = *fe;
        m.nonideal = 1;
        m.A = fe->A;
        m.B = fe->B;
        m.rho_c = fe->rho_c;
        m.kappa = fe->kappa;
        m.total = fe->total ? 1 : 0;
        m.model = fe->model;
    } else {
        m.nonideal = 0;
        m.rho_c = o.rho0;
    }
    c->sk_acc.assign(m.Q, nullptr);
    c->sk_count.assign(m.Q, 0);
    c->mv_sum.assign(m.Q, 0.0);

    if ((rc = alloc_guarded(c, &c->buf[0], c->pop_bytes(), "population buffer 0")) ||
        (rc = alloc_guarded(c, &c->buf[1], c->pop_bytes(), "population buffer 1")) ||
        (rc = alloc_guarded(c, &c->drho, c->field_bytes(), "density field")) || (rc = ensure_partials(c))) {
        free_all(c);
        delete c;
        return rc;
    }
    if (m.nonideal && m.model == 1 && m.kT > 0.0) {
        std::vector<double> chol(3 * (size_t)m.V);
        std::string err;
        if (!flb::swift_table(m, chol.data(), err)) {
            free_all(c);
            delete c;
            return fail(FLB_EINVAL, err);
        }
        if ((rc = alloc((void**)&c->sw_chol, chol.size() * sizeof(double))) ||
            (rc = alloc((void**)&c->sw_work, m.V * sizeof(double2))) ||
            (rc = alloc((void**)&c->sw_xi, m.V * sizeof(double2)))) {
            free_all(c);
            delete c;
            return rc;
        }
        const cudaError_t ce = cudaMemcpy(c->sw_chol, chol.data(), chol.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            free_all(c);
            delete c;
            return fail(FLB_ECUDA, std::string("uploading the noise table: ") + cudaGetErrorString(ce));
        }
        m.swift_xi = c->sw_xi;
    }
    // rest state: all deviations zero
    cudaError_t e = cudaMemsetAsync(c->buf[0], 0, c->pop_bytes(), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->buf[1], 0, c->pop_bytes(), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return fail(FLB_ECUDA, std::string("initialising the state: ") + cudaGetErrorString(e));
    }
    ztune_start(c);
    *out = c;
    return FLB_OK;
}

int flb_init(flb_ctx* c, const double* rho, const double* u, int thermal_init)
{
    FLB_TRACE();
    if (!c) return fail(FLB_EINVAL, "ctx is NULL");
    DeviceGuard guard(c->device);
    const HostModel& m = c->m;
    double* d_rho = nullptr;
    double* d_u = nullptr;
    int rc = FLB_OK;
    if (rho && (rc = alloc((void**)&d_rho, m.V * sizeof(double)))) return rc;
    if (u && (rc = alloc((void**)&d_u, (size_t)m.D * m.V * sizeof(double)))) {
        cudaFree(d_rho);
        return rc;
    }
    cudaError_t e = cudaSuccess;
    if (rho) e = cudaMemcpyAsync(d_rho, rho, m.V * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (u && e == cudaSuccess)
        e = cudaMemcpyAsync(d_u, u, (size_t)m.D * m.V * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = c->ops->init(m, c->buf[0], d_rho, d_u, thermal_init ? 1 : 0, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (d_rho) cudaFree(d_rho);
    if (d_u) cudaFree(d_u);
    if (e != cudaSuccess) return fail(FLB_ECUDA, std::string("flb_init: ") + cudaGetErrorString(e));
    c->cur = 0;
    c->step = 0;
    return flb_reset_accumulators(c);
}

// The time steps of flb_step; with dev_sums (device, 4 doubles per step) also
// the sums of the state each step starts from: the step kernel's own partial
// sums where it provides them, else the conservation reduction before the step
// (dev_sums[4 t] is the total mass: rho0 V is added to the summed deviations).
static int step_impl(flb_ctx* c, int nsteps, double* dev_sums)
{
    const double m0 = c->m.rho0 * (double)c->m.V;
    for (int t = 0; t < nsteps; ++t) {
        const void* src = c->buf[c->cur];
        void* dst = c->buf[c->cur ^ 1];
        size_t slot = 0;
        int rc;
        if (c->ops->step_needs_density(c->m)) {
            if ((rc = timer_begin(c, 0, &slot))) return rc;
            FLB_CUDA(c->ops->density(c->m, src, c->drho, c->stream));
            if (c->sw_xi)
                FLB_CUDA(flb::swift_noise(c->m, c->step, c->sw_chol, c->sw_work, c->sw_xi, c->prec != FLB_FP64,
                                          c->stream));
            if ((rc = timer_end(c, slot))) return rc;
        }
        if ((rc = timer_begin(c, 1, &slot))) return rc;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        const bool tune = c->zt.active && cudaStreamIsCapturing(c->stream, &cap) == cudaSuccess &&
                          cap == cudaStreamCaptureStatusNone;
        if (tune) {
            c->m.zchunk = c->zt.cand[c->zt.issued % c->zt.cand.size()];
            FLB_CUDA(cudaEventRecord(c->zt.ev[2 * c->zt.issued], c->stream));
        }
        cudaError_t se;
        if (dev_sums) {
            int nrows = 0;
            se = c->ops->step_rows(c->m, c->step, src, dst, c->drho, c->partials, &nrows, c->stream);
            if (se == cudaErrorNotSupported) {
                // this step kernel has no partial sums: reduce the state first
                FLB_CUDA(c->ops->cons_partials(c->m, src, c->partials, &nrows, c->stream));
                FLB_CUDA(flb::sum_columns(c->partials, nrows, 4, dev_sums + 4 * (size_t)t, c->stream, m0));
                se = c->ops->step(c->m, c->step, src, dst, c->drho, c->stream);
            } else if (se == cudaSuccess) {
                se = flb::sum_columns(c->partials, nrows, 4, dev_sums + 4 * (size_t)t, c->stream, m0);
            }
        } else {
            se = c->ops->step(c->m, c->step, src, dst, c->drho, c->stream);
        }
        if (tune) {
            c->m.zchunk = 0;
            FLB_CUDA(se);
            FLB_CUDA(cudaEventRecord(c->zt.ev[2 * c->zt.issued + 1], c->stream));
            if (++c->zt.issued == (int)(kZTuneRounds * c->zt.cand.size()) && (rc = ztune_finish(c))) return rc;
        }
        FLB_CUDA(se);
        if ((rc = timer_end(c, slot))) return rc;
        c->cur ^= 1;
        c->step += 1;
        if (c->check_every > 0 && c->step % (uint64_t)c->check_every == 0) {
            double s[4];
            if ((rc = timer_begin(c, 2, &slot))) return rc;
            rc = conservation(c, s);
            if (rc) return rc;
            if ((rc = timer_end(c, slot))) return rc;
            for (double v : s)
                if (!std::isfinite(v))
                    return fail(FLB_EDIVERGED, "non-finite mass or momentum at step " + std::to_string(c->step));
        }
        if (c->ev_used > 65536) {
            int r2 = timer_flush(c);
            if (r2) return r2;
        }
    }
    return FLB_OK;
}

int flb_step(flb_ctx* c, int nsteps)
{
    FLB_TRACE();
    if (!c) return fail(FLB_EINVAL, "ctx is NULL");
    if (nsteps < 0) return fail(FLB_EINVAL, "nsteps must be >= 0");
    DeviceGuard guard(c->device);
    return step_impl(c, nsteps, nullptr);
}

// Page-locked host memory that the device can address (cudaHostAlloc'd or
// registered memory under unified addressing): the column sums are written
// straight into it, with no copy on the stream.  NULL for other memory.
static double* device_alias(const double* host)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
        cudaGetLastError();  // pageable memory may report an error: not an alias
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost && at.devicePointer ? static_cast<double*>(at.devicePointer) : nullptr;
}

// The steps with their sums into `sums` (host): written in place when the
// device can address it, else staged on the device and copied on the stream.
static int step_sums_to_host(flb_ctx* c, int nsteps, double* sums)
{
    int rc = ensure_partials(c);
    if (rc) return rc;
    if (double* alias = device_alias(sums)) return step_impl(c, nsteps, alias);
    if ((size_t)nsteps > c->ss_cap) {
        if (c->ss_dev) cudaFree(c->ss_dev);
        c->ss_dev = nullptr;
        c->ss_cap = 0;
        if ((rc = alloc((void**)&c->ss_dev, 4 * (size_t)nsteps * sizeof(double)))) return rc;
        c->ss_cap = (size_t)nsteps;
    }
    if ((rc = step_impl(c, nsteps, c->ss_dev))) return rc;
    FLB_CUDA(cudaMemcpyAsync(sums, c->ss_dev, 4 * (size_t)nsteps * sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
    return FLB_OK;
}

int flb_step_sums_async(flb_ctx* c, int nsteps, double* sums)
{
    FLB_TRACE();
    if (!c) return fail(FLB_EINVAL, "ctx is NULL");
    if (nsteps < 0) return fail(FLB_EINVAL, "nsteps must be >= 0");
    if (nsteps > 0 && !sums) return fail(FLB_EINVAL, "sums is NULL");
    if (nsteps == 0) return FLB_OK;
    DeviceGuard guard(c->device);
    return step_sums_to_host(c, nsteps, sums);
}

int flb_step_sums(flb_ctx* c, int nsteps, double* sums)
{
    FLB_TRACE();
    if (!c) return fail(FLB_EINVAL, "ctx is NULL");
    if (nsteps < 0) return fail(FLB_EINVAL, "nsteps must be >= 0");
    if (nsteps > 0 && !sums) return fail(FLB_EINVAL, "sums is NULL");
    if (nsteps == 0) return FLB_OK;
    DeviceGuard guard(c->device);
    int rc = step_sums_to_host(c, nsteps, sums);
    if (rc) return rc;
    FLB_CUDA(cudaStreamSynchronize(c->stream));
    return FLB_OK;
}

int flb_moments(flb_ctx* c, double* out, int which)
{
    FLB_TRACE();
    if (!c || !out) return fail(FLB_EINVAL, "ctx or out is NULL");
    DeviceGuard guard(c->device);
    const HostModel& m = c->m;
    const void* src = c->buf[c->cur];
    if (which == FLB_MODE_VAR) {
        int rc = ensure_partials(c);
        if (rc) return rc;
        int nrows = 0;
        FLB_CUDA(c->ops->mode_partials(m, src, c->partials, &nrows, c->stream));
        std::vector<double> h(2 * m.Q);
        rc = reduce_to_host(c, nrows, 2 * m.Q, h.data());
        if (rc) return rc;
        c->mv_count += 1;
        for (int a = 0; a < m.Q; ++a) {
            const double mean = h[a] / (double)m.V;
            c->mv_sum[a] += h[m.Q + a] / (double)m.V - mean * mean;
            out[a] = c->mv_sum[a] / c->mv_count;
        }
        return FLB_OK;
    }
    if (which != FLB_RHO && which != FLB_U && which != FLB_MODES) return fail(FLB_EINVAL, "unknown observable");
    const size_t n = (which == FLB_RHO ? 1 : which == FLB_U ? m.D : m.Q) * (size_t)m.V;
    double* d_out = nullptr;
    int rc = alloc((void**)&d_out, n * sizeof(double));
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    const void* F = nullptr;
    if (which == FLB_U && m.nonideal && m.model == 0) {
        if ((rc = alloc(&c->mu, c->field_bytes())) || (rc = alloc(&c->F, 3 * c->field_bytes()))) {
            cudaFree(d_out);
            return rc;
        }
        e = c->ops->density(m, src, c->drho, c->stream);
        if (e == cudaSuccess) e = c->ops->mu_force(m, c->drho, c->mu, c->F, c->stream);
        F = c->F;
    }
    if (e == cudaSuccess) e = c->ops->moments(m, src, d_out, which, F, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_out);
    if (e != cudaSuccess) return fail(FLB_ECUDA, std::string("flb_moments: ") + cudaGetErrorString(e));
    return FLB_OK;
}

int flb_structure_factor(flb_ctx* c, double* S, int mode, int accumulate)
{
    FLB_TRACE();
    if (!c) return fail(FLB_EINVAL, "ctx is NULL");
    const HostModel& m = c->m;
    if (mode < 0 || mode >= m.Q) return fail(FLB_EINVAL, "mode out of range");
    DeviceGuard guard(c->device);
    int rc;
    if ((rc = alloc((void**)&c->fft, m.V * sizeof(double2))) || (rc = alloc((void**)&c->fft_scratch, m.V * sizeof(double2))))
        return rc;
    double* target = nullptr;
    if (accumulate) {
        if ((rc = alloc((void**)&c->sk_acc[mode], m.V * sizeof(double)))) return rc;
        if (c->sk_count[mode] == 0) FLB_CUDA(cudaMemsetAsync(c->sk_acc[mode], 0, m.V * sizeof(double), c->stream));
        target = c->sk_acc[mode];
    } else {
        if ((rc = alloc((void**)&c->sk_tmp, m.V * sizeof(double)))) return rc;
    }
    // single-precision states are transformed in single precision (GB300's
    // FP64 rate is a small fraction of its FP32 rate); |F|^2 accumulates in FP64
    const bool fp32 = c->prec != FLB_FP64;
    FLB_CUDA(c->ops->mode_field(m, c->buf[c->cur], mode, c->fft, fp32, c->stream));
    if (fp32) {
        FLB_CUDA(flb::fft3d((float2*)c->fft, m.X, m.Y, m.Z, (float2*)c->fft_scratch, c->stream));
        FLB_CUDA(flb::power_spectrum((const float2*)c->fft, m.V, target, c->sk_tmp, c->stream));
    } else {
        FLB_CUDA(flb::fft3d(c->fft, m.X, m.Y, m.Z, c->fft_scratch, c->stream));
        FLB_CUDA(flb::power_spectrum(c->fft, m.V, target, c->sk_tmp, c->stream));
    }
    if (accumulate) c->sk_count[mode] += 1;
    if (S) {
        const double* src = c->sk_tmp;
        if (accumulate) {
            // the mean over the snapshots, formed on the device
            if ((rc = alloc((void**)&c->sk_tmp, m.V * sizeof(double)))) return rc;
            FLB_CUDA(flb::scale_copy(c->sk_acc[mode], 1.0 / c->sk_count[mode], m.V, c->sk_tmp, c->stream));
            src = c->sk_tmp;
        }
        FLB_CUDA(cudaMemcpyAsync(S, src, m.V * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        FLB_CUDA(cudaStreamSynchronize(c->stream));
    }
    return FLB_OK;
}

int flb_snapshot_count(flb_ctx* c, int mode, int* count)
{
    if (!c || !count) return fail(FLB_EINVAL, "ctx or count is NULL");
    if (mode == -1) {
        *count = c->mv_count;
        return FLB_OK;
    }
    if (mode == -2) {
        *count = c->hs_count;
        return FLB_OK;
    }
    if (mode < 0 || mode >= c->m.Q) return fail(FLB_EINVAL, "mode out of range");
    *count = c->sk_count[mode];
    return FLB_OK;
}

int flb_reset_accumulators(flb_ctx* c)
{
    if (!c) return fail(FLB_EINVAL, "ctx is NULL");
    for (auto& n : c->sk_count) n = 0;
    for (auto& v : c->mv_sum) v = 0.0;
    c->mv_count = 0;
    c->hs_count = 0;
    return FLB_OK;
}

namespace {

int check_fit(const flb_ctx* c, const flb_interface_fit* f)
{
    if (!f) return fail(FLB_EINVAL, "fit is NULL");
    if (c->m.Q != 9) return fail(FLB_EINVAL, "interface heights need a D2Q9 context");
    if (!(f->width > 0) || !std::isfinite(f->rho_l) || !std::isfinite(f->rho_v) || f->rho_l == f->rho_v)
        return fail(FLB_EINVAL, "fit: width must be > 0 and rho_l != rho_v");
    if (f->window < 1 || 2 * f->window + 1 > c->m.Y) return fail(FLB_EINVAL, "fit: window must be in [1, (Y-1)/2]");
    if (f->iterations < 1 || f->iterations > 100) return fail(FLB_EINVAL, "fit: iterations must be in [1, 100]");
    for (int i = 0; i < 2; ++i)
        if (!std::isfinite(f->guess[i]) || std::fabs(f->guess[i]) > 1e9) return fail(FLB_EINVAL, "fit: bad guess");
    return FLB_OK;
}

// Heights of the current state into c->h_dev.
int heights_device(flb_ctx* c, const flb_interface_fit* f)
{
    const HostModel& m = c->m;
    int rc;
    if ((rc = alloc((void**)&c->h_dev, 2 * (size_t)m.X * sizeof(double)))) return rc;
    FLB_CUDA(c->ops->density(m, c->buf[c->cur], c->drho, c->stream));
    FLB_CUDA(flb::interface_heights(c->drho, c->ops->real_size, m.rho0, m.X, m.Y, *f, c->h_dev, c->stream));
    return FLB_OK;
}

}  // namespace

int flb_interface_heights(flb_ctx* c, const flb_interface_fit* fit, double* h)
{
    FLB_TRACE();
    if (!c || !h) return fail(FLB_EINVAL, "ctx or h is NULL");
    int rc;
    if ((rc = check_fit(c, fit))) return rc;
    DeviceGuard guard(c->device);
    if ((rc = heights_device(c, fit))) return rc;
    FLB_CUDA(cudaMemcpyAsync(h, c->h_dev, 2 * (size_t)c->m.X * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    FLB_CUDA(cudaStreamSynchronize(c->stream));
    return FLB_OK;
}

int flb_height_spectrum(flb_ctx* c, const flb_interface_fit* fit, double* S, int accumulate)
{
    FLB_TRACE();
    if (!c) return fail(FLB_EINVAL, "ctx is NULL");
    int rc;
    if ((rc = check_fit(c, fit))) return rc;
    DeviceGuard guard(c->device);
    const int X = c->m.X;
    if ((rc = alloc((void**)&c->hs_work, 2 * (size_t)X * sizeof(double2))) ||
        (rc = alloc((void**)&c->hs_scratch, 2 * (size_t)X * sizeof(double2))) ||
        (rc = alloc((void**)&c->hs_acc, (size_t)X * sizeof(double))) ||
        (rc = alloc((void**)&c->hs_tmp, (size_t)X * sizeof(double))))
        return rc;
    if ((rc = heights_device(c, fit))) return rc;
    if (accumulate && c->hs_count == 0) FLB_CUDA(cudaMemsetAsync(c->hs_acc, 0, X * sizeof(double), c->stream));
    FLB_CUDA(flb::height_power(c->h_dev, X, c->hs_work, c->hs_scratch, accumulate ? c->hs_acc : nullptr, c->hs_tmp,
                               c->stream));
    if (accumulate) c->hs_count += 1;
    if (S) {
        FLB_CUDA(cudaMemcpyAsync(S, accumulate ? c->hs_acc : c->hs_tmp, X * sizeof(double), cudaMemcpyDeviceToHost,
                                 c->stream));
        FLB_CUDA(cudaStreamSynchronize(c->stream));
        if (accumulate) {
            const double inv = 1.0 / c->hs_count;
            for (int k = 0; k < X; ++k) S[k] *= inv;
        }
    }
    return FLB_OK;
}

int flb_z_chunk(flb_ctx* c, int* planes, int* tuning)
{
    if (!c || !planes || !tuning) return fail(FLB_EINVAL, "NULL argument");
    *planes = std::min(c->m.zchunk > 0 ? c->m.zchunk : flb::kZChunkDefault, c->m.Z);
    *tuning = c->zt.active ? 1 : 0;
    return FLB_OK;
}

int flb_check_guards(flb_ctx* c)
{
    if (!c) return fail(FLB_EINVAL, "ctx is NULL");
    if (c->guards.empty()) return fail(FLB_EINVAL, "the context was created without guard zones (opt.guard = 0)");
    DeviceGuard guard(c->device);
    FLB_CUDA(cudaStreamSynchronize(c->stream));
    std::vector<unsigned char> h(kGuardBytes);
    for (const auto& g : c->guards) {
        const char* zones[2] = {(const char*)g.base, (const char*)g.base + kGuardBytes + g.bytes};
        for (int side = 0; side < 2; ++side) {
            FLB_CUDA(cudaMemcpy(h.data(), zones[side], kGuardBytes, cudaMemcpyDeviceToHost));
            for (size_t k = 0; k < kGuardBytes; ++k)
                if (h[k] != kGuardByte) {
                    const long long off = side == 0 ? (long long)k - (long long)kGuardBytes : (long long)(g.bytes + k);
                    return fail(FLB_EBOUNDS, std::string("write outside the ") + g.name + " (" +
                                                 (side == 0 ? "before its start" : "after its end") +
                                                 "): first changed byte at offset " + std::to_string(off));
                }
        }
    }
    return FLB_OK;
}

int flb_conservation(flb_ctx* c, double out[4])
{
    FLB_TRACE();
    if (!c || !out) return fail(FLB_EINVAL, "ctx or out is NULL");
    DeviceGuard guard(c->device);
    return conservation(c, out);
}

int flb_get_populations(flb_ctx* c, double* f)
{
    FLB_TRACE();
    if (!c || !f) return fail(FLB_EINVAL, "ctx or f is NULL");
    DeviceGuard guard(c->device);
    const size_t n = (size_t)c->m.Q * c->m.V;
    double* d = nullptr;
    int rc = alloc((void**)&d, n * sizeof(double));
    if (rc) return rc;
    cudaError_t e = c->ops->get_pop(c->m, c->buf[c->cur], d, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(FLB_ECUDA, std::string("flb_get_populations: ") + cudaGetErrorString(e));
    return FLB_OK;
}

int flb_get_sites(flb_ctx* c, const long long* sites, int n, double* f)
{
    FLB_TRACE();
    if (!c) return fail(FLB_EINVAL, "ctx is NULL");
    if (n < 0) return fail(FLB_EINVAL, "n must be >= 0");
    if (n == 0) return FLB_OK;
    if (!sites || !f) return fail(FLB_EINVAL, "sites or f is NULL");
    for (int k = 0; k < n; ++k)
        if (sites[k] < 0 || sites[k] >= c->m.V)
            return fail(FLB_EINVAL, "site " + std::to_string(sites[k]) + " outside [0, V)");
    DeviceGuard guard(c->device);
    long long* d_sites = nullptr;
    double* d = nullptr;
    int rc = alloc((void**)&d_sites, (size_t)n * sizeof(long long));
    if (rc) return rc;
    if ((rc = alloc((void**)&d, (size_t)c->m.Q * n * sizeof(double)))) {
        cudaFree(d_sites);
        return rc;
    }
    cudaError_t e = cudaMemcpyAsync(d_sites, sites, (size_t)n * sizeof(long long), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = c->ops->get_sites(c->m, c->buf[c->cur], d_sites, n, d, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f, d, (size_t)c->m.Q * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    cudaFree(d_sites);
    if (e != cudaSuccess) return fail(FLB_ECUDA, std::string("flb_get_sites: ") + cudaGetErrorString(e));
    return FLB_OK;
}

int flb_set_populations(flb_ctx* c, const double* f)
{
    FLB_TRACE();
    if (!c || !f) return fail(FLB_EINVAL, "ctx or f is NULL");
    DeviceGuard guard(c->device);
    const size_t n = (size_t)c->m.Q * c->m.V;
    double* d = nullptr;
    int rc = alloc((void**)&d, n * sizeof(double));
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(d, f, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = c->ops->set_pop(c->m, d, c->buf[c->cur], c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(FLB_ECUDA, std::string("flb_set_populations: ") + cudaGetErrorString(e));
    return FLB_OK;
}

int flb_get_state_device(flb_ctx* c, void* g)
{
    FLB_TRACE();
    if (!c || !g) return fail(FLB_EINVAL, "ctx or g is NULL");
    DeviceGuard guard(c->device);
    FLB_CUDA(c->ops->pull_state(c->m, c->buf[c->cur], g, c->stream));
    return FLB_OK;
}

int flb_set_state_device(flb_ctx* c, const void* g)
{
    FLB_TRACE();
    if (!c || !g) return fail(FLB_EINVAL, "ctx or g is NULL");
    DeviceGuard guard(c->device);
    FLB_CUDA(c->ops->push_state(c->m, g, c->buf[c->cur], c->stream));
    return FLB_OK;
}

int flb_adjoint_step(flb_ctx* c, const void* g_n, uint64_t step, const void* lam_next, void* lam, double* grad)
{
    FLB_TRACE();
    if (!c || !g_n || !lam_next || !lam || !grad) return fail(FLB_EINVAL, "NULL argument");
    if (c->m.Q != 19) return fail(FLB_EINVAL, "the adjoint step is implemented for D3Q19");
    if (c->prec == FLB_BF16) return fail(FLB_EINVAL, "the adjoint step needs FLB_FP64 or FLB_FP32 storage");
    if (lam == lam_next) return fail(FLB_EINVAL, "lam and lam_next must not alias");
    DeviceGuard guard(c->device);
    int rc;
    if ((rc = alloc(&c->adj_work, 10 * c->field_bytes())) ||
        (rc = alloc((void**)&c->adj_rows, (size_t)flb::adjoint_rows(c->m) * 6 * sizeof(double))))
        return rc;
    FLB_CUDA(flb::adjoint_step(c->m, c->prec, step, g_n, lam_next, nullptr, lam, nullptr, c->adj_work, c->adj_rows,
                               grad, c->stream));
    return FLB_OK;
}

int flb_adjoint_segment(flb_ctx* c, const void* g_start, uint64_t step0, int n, void* states, void* lam,
                        double* grad)
{
    FLB_TRACE();
    if (!c || !g_start || !states || !lam || !grad) return fail(FLB_EINVAL, "NULL argument");
    if (n < 1) return fail(FLB_EINVAL, "n must be >= 1");
    if (c->m.Q != 19) return fail(FLB_EINVAL, "the adjoint step is implemented for D3Q19");
    if (c->prec == FLB_BF16) return fail(FLB_EINVAL, "the adjoint step needs FLB_FP64 or FLB_FP32 storage");
    DeviceGuard guard(c->device);
    int rc;
    if ((rc = alloc(&c->adj_work, 10 * c->field_bytes())) ||
        (rc = alloc((void**)&c->adj_rows, (size_t)flb::adjoint_rows(c->m) * 6 * sizeof(double))) ||
        (rc = alloc(&c->adj_lam2, c->pop_bytes())) ||
        (rc = alloc(&c->adj_rb, 2 * c->field_bytes())))
        return rc;
    const size_t pb = c->pop_bytes();
    char* S = (char*)states;
    // forward: the states at step0 .. step0+n-1 (pre-collision deviations)
    FLB_CUDA(cudaMemcpyAsync(S, g_start, pb, cudaMemcpyDeviceToDevice, c->stream));
    FLB_CUDA(c->ops->push_state(c->m, g_start, c->buf[c->cur], c->stream));
    c->step = step0;
    for (int k = 1; k < n; ++k) {
        if ((rc = flb_step(c, 1))) return rc;
        FLB_CUDA(c->ops->pull_state(c->m, c->buf[c->cur], S + (size_t)k * pb, c->stream));
    }
    // reverse: lam(step0 + n) -> lam(step0), alternating between lam and
    // adj_lam2; for the non-ideal fluid each step passes its density part on to
    // the next (two scalars per site instead of a pass over all 19 planes) and
    // the last one is added at the end, the same additions in the same order
    // as flb_adjoint_step one step at a time
    void* nxt = lam;
    void* cur = c->adj_lam2;
    char* rb = (char*)c->adj_rb;
    const size_t fb = c->field_bytes();
    const bool defer = c->m.nonideal != 0;
    const void* rb_in = nullptr;
    for (int k = n - 1; k >= 0; --k) {
        void* rb_out = defer ? rb + (size_t)(k & 1) * fb : nullptr;
        FLB_CUDA(flb::adjoint_step(c->m, c->prec, step0 + (uint64_t)k, S + (size_t)k * pb, nxt, rb_in, cur, rb_out,
                                   c->adj_work, c->adj_rows, grad, c->stream));
        rb_in = rb_out;
        std::swap(nxt, cur);
    }
    if (rb_in) FLB_CUDA(flb::adjoint_add_rb(c->m, c->prec, nxt, rb_in, c->stream));
    if (nxt != lam) FLB_CUDA(cudaMemcpyAsync(lam, nxt, pb, cudaMemcpyDeviceToDevice, c->stream));
    return FLB_OK;
}

int flb_get_step(flb_ctx* c, uint64_t* step)
{
    if (!c || !step) return fail(FLB_EINVAL, "ctx or step is NULL");
    *step = c->step;
    return FLB_OK;
}

int flb_set_step(flb_ctx* c, uint64_t step)
{
    if (!c) return fail(FLB_EINVAL, "ctx is NULL");
    c->step = step;
    return FLB_OK;
}

int flb_set_stream(flb_ctx* c, void* stream)
{
    if (!c) return fail(FLB_EINVAL, "ctx is NULL");
    DeviceGuard guard(c->device);
    int rc = timer_flush(c);
    if (rc) return rc;
    FLB_CUDA(cudaStreamSynchronize(c->stream));
    c->stream = (cudaStream_t)stream;
    return FLB_OK;
}

int flb_synchronize(flb_ctx* c)
{
    if (!c) return fail(FLB_EINVAL, "ctx is NULL");
    DeviceGuard guard(c->device);
    FLB_CUDA(cudaStreamSynchronize(c->stream));
    return FLB_OK;
}

int flb_get_info(flb_ctx* c, int out[6])
{
    if (!c || !out) return fail(FLB_EINVAL, "ctx or out is NULL");
    out[0] = c->m.Q;
    out[1] = c->m.D;
    out[2] = c->m.X;
    out[3] = c->m.Y;
    out[4] = c->m.Z;
    out[5] = c->prec;
    return FLB_OK;
}

int flb_kernel_timing(flb_ctx* c, int enable)
{
    if (!c) return fail(FLB_EINVAL, "ctx is NULL");
    DeviceGuard guard(c->device);
    int rc = timer_flush(c);
    if (rc) return rc;
    c->timing = enable != 0;
    for (int k = 0; k < FLB_NKERNEL_TIMERS; ++k) {
        c->t_ms[k] = 0.0;
        c->t_n[k] = 0;
    }
    return FLB_OK;
}

int flb_kernel_times(flb_ctx* c, double* ms, int* launches)
{
    if (!c || !ms || !launches) return fail(FLB_EINVAL, "NULL argument");
    DeviceGuard guard(c->device);
    int rc = timer_flush(c);
    if (rc) return rc;
    for (int k = 0; k < FLB_NKERNEL_TIMERS; ++k) {
        ms[k] = c->t_ms[k];
        launches[k] = c->t_n[k];
    }
    return FLB_OK;
}

int flb_save(flb_ctx* c, const char* path)
{
    FLB_TRACE();
    if (!c || !path) return fail(FLB_EINVAL, "ctx or path is NULL");
    DeviceGuard guard(c->device);
    std::vector<char> host(c->pop_bytes());
    FLB_CUDA(cudaMemcpyAsync(host.data(), c->buf[c->cur], host.size(), cudaMemcpyDeviceToHost, c->stream));
    FLB_CUDA(cudaStreamSynchronize(c->stream));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(FLB_EIO, std::string("cannot open ") + path);
    const HostModel& m = c->m;
    // ints[7]: free-energy flags, total | model << 1
    const int32_t ints[8] = {m.Q, m.X, m.Y, m.Z, c->prec, c->fe.enabled, m.noise_local,
                             (c->fe.total ? 1 : 0) | (c->fe.model << 1)};
    const double dbl[10] = {m.rho0, m.om_s, m.om_b, m.om_g, m.kT, c->fe.A, c->fe.B, c->fe.rho_c, c->fe.kappa, 0.0};
    const uint64_t u64[3] = {m.seed, (uint64_t)m.replica, c->step};
    bool ok = std::fwrite(kMagic, 1, 8, fp) == 8 && std::fwrite(ints, sizeof(ints), 1, fp) == 1 &&
              std::fwrite(dbl, sizeof(dbl), 1, fp) == 1 && std::fwrite(u64, sizeof(u64), 1, fp) == 1 &&
              std::fwrite(host.data(), 1, host.size(), fp) == host.size();
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? FLB_OK : fail(FLB_EIO, std::string("short write to ") + path);
}

int flb_load(flb_ctx** out, const char* path, const flb_options* opt)
{
    FLB_TRACE();
    if (!out || !path) return fail(FLB_EINVAL, "out or path is NULL");
    *out = nullptr;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(FLB_EIO, std::string("cannot open ") + path);
    char magic[8];
    int32_t ints[8];
    double dbl[10];
    uint64_t u64[3];
    bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(ints, sizeof(ints), 1, fp) == 1 && std::fread(dbl, sizeof(dbl), 1, fp) == 1 &&
              std::fread(u64, sizeof(u64), 1, fp) == 1;
    if (!ok) {
        std::fclose(fp);
        return fail(FLB_EIO, std::string("not an flb checkpoint: ") + path);
    }
    flb_options o;
    flb_default_options(&o);
    if (opt) o = *opt;
    o.precision = ints[4];
    o.rho0 = dbl[0];
    o.replica = (uint32_t)u64[1];
    o.noise_rho_local = ints[6];
    flb_free_energy fe{ints[5], dbl[5], dbl[6], dbl[7], dbl[8], ints[7] & 1, (ints[7] >> 1) & 1};
    const int dims[3] = {ints[1], ints[2], ints[3]};
    flb_ctx* c = nullptr;
    int rc = flb_create(&c, ints[0], dims, dbl[1], dbl[2], dbl[3], dbl[4], &fe, u64[0], &o);
    if (rc) {
        std::fclose(fp);
        return rc;
    }
    std::vector<char> host(c->pop_bytes());
    ok = std::fread(host.data(), 1, host.size(), fp) == host.size();
    std::fclose(fp);
    if (!ok) {
        flb_destroy(c);
        return fail(FLB_EIO, std::string("truncated checkpoint: ") + path);
    }
    {
        DeviceGuard guard(c->device);
        cudaError_t e = cudaMemcpyAsync(c->buf[0], host.data(), host.size(), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            flb_destroy(c);
            return fail(FLB_ECUDA, std::string("flb_load: ") + cudaGetErrorString(e));
        }
    }
    c->cur = 0;
    c->step = u64[2];
    *out = c;
    return FLB_OK;
}

const char* flb_error_string(int code)
{
    switch (code) {
    case FLB_OK: return "success";
    case FLB_EINVAL: return "invalid argument";
    case FLB_ENOMEM: return "out of memory";
    case FLB_ECUDA: return "CUDA error";
    case FLB_EDIVERGED: return "simulation diverged (non-finite mass or momentum)";
    case FLB_ETIMEOUT: return "device wait timed out";
    case FLB_EIO: return "checkpoint I/O error";
    case FLB_EBOUNDS: return "write outside a device buffer (guard zone overwritten)";
    default: return "unknown error";
    }
}

const char* flb_last_error(void) { return g_last_error.c_str(); }

void flb_destroy(flb_ctx* c)
{
    if (!c) return;
    DeviceGuard guard(c->device);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"
