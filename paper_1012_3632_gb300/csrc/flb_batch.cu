// flb_batch.cu -- many independent fluctuating ideal-gas D3Q19 lattices of
// uneven sizes advanced together (ensemble averages for the FDT statistics of
// Sec. VI).  One persistent kernel per time step walks a flattened work list
// of (replica, tile) items; per-replica sizes, relaxation rates, noise scales
// and Philox keys live in the kernel's parameter bank; the time step index
// lives in device memory so that a CUDA graph of two steps can be replayed.
// A small autotuner picks the tile shape per lattice size.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/flb.h"
#include "flb_internal.h"
#include "flb_kernels.cuh"

namespace flb {

// Collision parameters of one replica (flb_fp32.cu).
Coll<float> coll_fp32(const HostModel& m, uint64_t step);

namespace {

// Tile shapes (x, y, z), 256 sites each, powers of two (x at least 2: one
// site pair per thread along x).
constexpr int kShapes[][3] = {{32, 8, 1}, {32, 4, 2}, {32, 2, 4}, {16, 16, 1}, {16, 8, 2}, {16, 4, 4}, {8, 8, 4},
                              {64, 4, 1}, {64, 2, 2}, {64, 1, 4}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

struct BatchRep {
    int X, Y, Z;
    int lx, ly;          // log2 of the tile's x and y extent
    int tx, ty, tz;      // tile extent
    long long off;       // element offset of the replica's populations in each arena
    Coll<float> c;
};

struct BatchArgs {
    int n;
    const float* src;
    float* dst;
    BatchRep rep[FLB_BATCH_MAX];
};
static_assert(sizeof(BatchArgs) < 32000, "batch parameters exceed the kernel parameter space");

// Work item: replica and tile coordinates.
struct Tile {
    int r, bx, by, bz;
};

// 128 threads per tile of tx*ty*tz = 256 sites: one thread per site pair
// (x, x+1) along x when the replica's X is even (packed FP32 arithmetic, as the
// single-lattice kernel k_step2), otherwise one site per thread in two passes.
// OFF32: every replica has 19 V < 2^31, so a population's element offset from
// its replica's base fits in 32 bits (one address operation per access).
template <bool OFF32>
__global__ void __launch_bounds__(128) k_step_batch(const __grid_constant__ BatchArgs A, const int4* __restrict__ tiles,
                                                    int ntiles, const unsigned long long* __restrict__ d_step)
{
    using Off = typename std::conditional<OFF32, int, long>::type;
    using L = D3Q19;
    const uint32_t step = (uint32_t)__ldg(d_step);
    // the next work item is fetched one iteration ahead, off the path of the pulls
    int4 w_next = (int)blockIdx.x < ntiles ? __ldg(tiles + blockIdx.x) : make_int4(0, 0, 0, 0);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 w = w_next;
        if (t + (int)gridDim.x < ntiles) w_next = __ldg(tiles + t + gridDim.x);
        const BatchRep& B = A.rep[w.x];
        const float* src = A.src + B.off;
        float* dst = A.dst + B.off;
        const int X = B.X, Y = B.Y, Z = B.Z;
        const Off V = (Off)X * Y * Z;
        if ((X & 1) == 0) {
            const int hx = B.tx >> 1;  // pairs per tile row
            const int x = w.y * B.tx + 2 * (threadIdx.x & (hx - 1));
            const int y = w.z * B.ty + ((threadIdx.x >> (B.lx - 1)) & (B.ty - 1));
            const int z = w.w * B.tz + (threadIdx.x >> (B.lx - 1 + B.ly));
            if (x >= X || y >= Y || z >= Z) continue;
            const int xm = x == 0 ? X - 1 : x - 1, x2 = x + 2 == X ? 0 : x + 2;
            const int yv[3] = {wrap_once(y - 1, Y), y, wrap_once(y + 1, Y)};
            const int zv[3] = {wrap_once(z - 1, Z), z, wrap_once(z + 1, Z)};
            F2 g[L::Q];
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const float* p = src + ((Off)i * V + X * (yv[1 - Vel<L>::cy(i)] + Y * zv[1 - Vel<L>::cz(i)]));
                const int cx = Vel<L>::cx(i);
                if (cx == 0)
                    g[i] = mk2(ld_stream2(p + x));
                else if (cx > 0)
                    g[i] = F2(ld_stream1(p + xm), ld_stream1(p + x));
                else
                    g[i] = F2(ld_stream1(p + x + 1), ld_stream1(p + x2));
            }
            const int s = x + X * (y + Y * z);
            L::template collide<false, true>(g, F2(0.f), F2(0.f), F2(0.f), B.c, (uint32_t)s, step);
#pragma unroll
            for (int i = 0; i < L::Q; ++i) __stcs(reinterpret_cast<float2*>(dst + ((Off)i * V + s)), g[i].v);
        } else {
            for (int half = 0; half < 2; ++half) {
                const int q = threadIdx.x + 128 * half;
                const int x = w.y * B.tx + (q & (B.tx - 1));
                const int y = w.z * B.ty + ((q >> B.lx) & (B.ty - 1));
                const int z = w.w * B.tz + (q >> (B.lx + B.ly));
                if (x >= X || y >= Y || z >= Z) continue;
                const Nbhd nb(x, y, z, X, Y, Z);
                float g[L::Q];
#pragma unroll
                for (int i = 0; i < L::Q; ++i)
                    g[i] = src[(Off)i * V + nb.src(Vel<L>::cx(i), Vel<L>::cy(i), Vel<L>::cz(i))];
                const int s = x + X * (y + Y * z);
                L::template collide<false>(g, 0.f, 0.f, 0.f, B.c, (uint32_t)s, step);
#pragma unroll
                for (int i = 0; i < L::Q; ++i) __stcs(dst + ((Off)i * V + s), g[i]);
            }
        }
    }
}

__global__ void k_advance(unsigned long long* d_step) { *d_step += 1ull; }

int ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

}  // namespace
}  // namespace flb

using flb::BatchArgs;
using flb::BatchRep;
using flb::HostModel;

struct flb_batch {
    int n = 0;
    int device = 0;
    cudaStream_t stream = nullptr;    // caller's stream
    cudaStream_t cap = nullptr;       // internal stream used for graph capture
    std::vector<HostModel> m;         // per replica
    std::vector<long long> off;       // element offset per replica
    std::vector<int> shape;           // index into kShapes per replica
    long long total = 0;              // elements per arena
    long long sites = 0;
    float* buf[2] = {nullptr, nullptr};
    int cur = 0;
    unsigned long long* d_step = nullptr;
    uint64_t step = 0;
    int4* tiles = nullptr;
    int ntiles = 0;
    int grid = 0;
    bool off32 = true;                // every replica: 19 V < 2^31 (k_step_batch<true>)
    BatchArgs args[2];                // src/dst for cur = 0 and cur = 1
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    // reductions
    double* partials = nullptr;
    double* red = nullptr;
    std::vector<double> mv_sum;       // n * Q
    int mv_count = 0;
    double2* fft = nullptr;
    double2* fft_scratch = nullptr;
    double* sk_tmp = nullptr;
    std::map<std::pair<int, int>, std::pair<double*, int>> sk_acc;  // (replica, mode) -> (acc, count)
};

namespace {

int bfail(int code, const std::string& msg) { return flb::set_error(code, msg); }

#define BCUDA(call)                                                                                       \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return bfail(e_ == cudaErrorMemoryAllocation ? FLB_ENOMEM : FLB_ECUDA,                        \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                             \
    } while (0)

struct Dev {
    int prev = -1;
    explicit Dev(int d)
    {
        cudaGetDevice(&prev);
        if (d != prev) cudaSetDevice(d);
    }
    ~Dev()
    {
        int c = -1;
        if (prev >= 0 && cudaGetDevice(&c) == cudaSuccess && c != prev) cudaSetDevice(prev);
    }
};

void drop_graphs(flb_batch* b)
{
    for (auto& g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Rebuild the work list and the kernel parameters after a shape change.
int build_tiles(flb_batch* b)
{
    std::vector<int4> t;
    for (int r = 0; r < b->n; ++r) {
        const int* sh = flb::kShapes[b->shape[r]];
        const HostModel& m = b->m[r];
        const int nx = (m.X + sh[0] - 1) / sh[0], ny = (m.Y + sh[1] - 1) / sh[1], nz = (m.Z + sh[2] - 1) / sh[2];
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) t.push_back(make_int4(r, i, j, k));
    }
    if (b->tiles) cudaFree(b->tiles);
    b->tiles = nullptr;
    b->ntiles = (int)t.size();
    BCUDA(cudaMalloc(&b->tiles, t.size() * sizeof(int4)));
    BCUDA(cudaMemcpy(b->tiles, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice));
    for (int p = 0; p < 2; ++p) {
        BatchArgs& A = b->args[p];
        std::memset(&A, 0, sizeof(A));
        A.n = b->n;
        A.src = b->buf[p];
        A.dst = b->buf[p ^ 1];
        for (int r = 0; r < b->n; ++r) {
            const int* sh = flb::kShapes[b->shape[r]];
            BatchRep& R = A.rep[r];
            R.X = b->m[r].X;
            R.Y = b->m[r].Y;
            R.Z = b->m[r].Z;
            R.tx = sh[0];
            R.ty = sh[1];
            R.tz = sh[2];
            R.lx = flb::ilog2(sh[0]);
            R.ly = flb::ilog2(sh[1]);
            R.off = b->off[r];
            R.c = flb::coll_fp32(b->m[r], 0);
        }
    }
    drop_graphs(b);
    return FLB_OK;
}

int launch_step(flb_batch* b, cudaStream_t st)
{
    if (b->off32)
        flb::k_step_batch<true><<<b->grid, 128, 0, st>>>(b->args[b->cur], b->tiles, b->ntiles, b->d_step);
    else
        flb::k_step_batch<false><<<b->grid, 128, 0, st>>>(b->args[b->cur], b->tiles, b->ntiles, b->d_step);
    flb::k_advance<<<1, 1, 0, st>>>(b->d_step);
    BCUDA(cudaGetLastError());
    return FLB_OK;
}

// Graph of two steps starting from buffer parity p (ends at parity p).
int make_graph(flb_batch* b, int p)
{
    if (b->graph[p]) return FLB_OK;
    cudaGraph_t g = nullptr;
    BCUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    const int save = b->cur;
    b->cur = p;
    int rc = launch_step(b, b->cap);
    b->cur = p ^ 1;
    if (!rc) rc = launch_step(b, b->cap);
    b->cur = save;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return bfail(FLB_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph[p], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(FLB_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return FLB_OK;
}

const float* rep_src(const flb_batch* b, int r) { return b->buf[b->cur] + b->off[r]; }

}  // namespace

extern "C" {

int flb_batch_create(flb_batch** out, int lattice, int n, const int* dims, const double* omega_shear,
                     const double* omega_bulk, const double* omega_ghost, const double* kT, const uint64_t* seeds,
                     const flb_options* opt)
{
    FLB_TRACE();
    if (!out) return bfail(FLB_EINVAL, "out is NULL");
    *out = nullptr;
    if (lattice != FLB_D3Q19) return bfail(FLB_EINVAL, "batches support FLB_D3Q19");
    if (n < 1 || n > FLB_BATCH_MAX) return bfail(FLB_EINVAL, "n must be in [1, FLB_BATCH_MAX]");
    if (!dims || !omega_shear || !kT || !seeds) return bfail(FLB_EINVAL, "NULL argument");
    flb_options o;
    flb_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != FLB_FP32) return bfail(FLB_EINVAL, "batches store populations in FLB_FP32");
    if (!(o.rho0 > 0.0)) return bfail(FLB_EINVAL, "rho0 must be positive");
    for (int r = 0; r < n; ++r) {
        for (int d = 0; d < 3; ++d)
            if (dims[3 * r + d] < 1) return bfail(FLB_EINVAL, "every dimension must be >= 1");
        const double oms[3] = {omega_shear[r], omega_bulk ? omega_bulk[r] : 1.0, omega_ghost ? omega_ghost[r] : 1.0};
        for (double om : oms)
            if (!(om > 0.0 && om < 2.0)) return bfail(FLB_EINVAL, "relaxation rates must lie in (0, 2)");
        if (!(kT[r] >= 0.0 && kT[r] <= o.rho0 / 3.0)) return bfail(FLB_EINVAL, "kT must lie in [0, cs^2 rho0]");
        if ((double)dims[3 * r] * dims[3 * r + 1] * dims[3 * r + 2] >= 2147483648.0)
            return bfail(FLB_EINVAL, "replica too large");
    }
    flb_batch* b = new (std::nothrow) flb_batch();
    if (!b) return bfail(FLB_ENOMEM, "host allocation failed");
    int dev = o.device;
    if (dev < 0) cudaGetDevice(&dev);
    b->device = dev;
    Dev guard(dev);
    b->n = n;
    b->stream = (cudaStream_t)o.stream;
    b->m.resize(n);
    b->off.resize(n);
    b->shape.assign(n, 0);
    for (int r = 0; r < n; ++r) {
        HostModel& m = b->m[r];
        m.Q = 19;
        m.D = 3;
        m.X = dims[3 * r];
        m.Y = dims[3 * r + 1];
        m.Z = dims[3 * r + 2];
        m.V = (long)m.X * m.Y * m.Z;
        m.rho0 = o.rho0;
        m.om_s = omega_shear[r];
        m.om_b = omega_bulk ? omega_bulk[r] : 1.0;
        m.om_g = omega_ghost ? omega_ghost[r] : 1.0;
        m.kT = kT[r];
        m.nonideal = 0;
        m.rho_c = o.rho0;
        m.seed = seeds[r];
        m.replica = o.replica + (uint32_t)r;
        m.noise_local = o.noise_rho_local ? 1 : 0;
        b->off[r] = b->total;
        b->total += 19LL * m.V;
        b->sites += m.V;
        if (19LL * m.V >= (1LL << 31)) b->off32 = false;
        b->shape[r] = (m.X % 32 == 0) ? 1 : 4;  // (32,4,2) or (16,8,2) until tuned
    }
    b->mv_sum.assign((size_t)n * 19, 0.0);
    int rc = FLB_OK;
    auto cleanup = [&](int code) {
        flb_batch_destroy(b);
        return code;
    };
    cudaError_t e = cudaMalloc(&b->buf[0], b->total * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b->buf[1], b->total * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_step, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(b->buf[0], 0, b->total * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(b->buf[1], 0, b->total * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(b->d_step, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess)
        return cleanup(bfail(e == cudaErrorMemoryAllocation ? FLB_ENOMEM : FLB_ECUDA,
                             std::string("flb_batch_create: ") + cudaGetErrorString(e)));
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    if (b->off32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, flb::k_step_batch<true>, 128, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, flb::k_step_batch<false>, 128, 0);
    b->grid = std::max(1, nsm * std::max(1, per_sm));
    if ((rc = build_tiles(b))) return cleanup(rc);
    *out = b;
    return FLB_OK;
}

int flb_batch_init(flb_batch* b, int thermal_init)
{
    FLB_TRACE();
    if (!b) return bfail(FLB_EINVAL, "batch is NULL");
    Dev guard(b->device);
    const flb::PrecOps& ops = flb::ops_fp32();
    for (int r = 0; r < b->n; ++r)
        BCUDA(ops.init(b->m[r], b->buf[0] + b->off[r], nullptr, nullptr, thermal_init ? 1 : 0, b->stream));
    BCUDA(cudaMemsetAsync(b->d_step, 0, sizeof(unsigned long long), b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    b->cur = 0;
    b->step = 0;
    b->mv_count = 0;
    std::fill(b->mv_sum.begin(), b->mv_sum.end(), 0.0);
    for (auto& kv : b->sk_acc) kv.second.second = 0;
    return FLB_OK;
}

int flb_batch_step(flb_batch* b, int nsteps)
{
    FLB_TRACE();
    if (!b) return bfail(FLB_EINVAL, "batch is NULL");
    if (nsteps < 0) return bfail(FLB_EINVAL, "nsteps must be >= 0");
    Dev guard(b->device);
    int rc;
    int left = nsteps;
    if (left >= 2) {
        if ((rc = make_graph(b, b->cur))) return rc;
        while (left >= 2) {
            BCUDA(cudaGraphLaunch(b->graph[b->cur], b->stream));
            left -= 2;
        }
    }
    if (left == 1) {
        if ((rc = launch_step(b, b->stream))) return rc;
        b->cur ^= 1;
    }
    b->step += (uint64_t)nsteps;
    return FLB_OK;
}

int flb_batch_autotune(flb_batch* b, int* shapes_out)
{
    FLB_TRACE();
    if (!b) return bfail(FLB_EINVAL, "batch is NULL");
    Dev guard(b->device);
    // distinct lattice sizes
    std::map<std::vector<int>, std::vector<int>> groups;
    for (int r = 0; r < b->n; ++r) groups[{b->m[r].X, b->m[r].Y, b->m[r].Z}].push_back(r);
    cudaEvent_t e0, e1;
    BCUDA(cudaEventCreate(&e0));
    BCUDA(cudaEventCreate(&e1));
    const std::vector<int> saved = b->shape;
    int rc = FLB_OK;
    for (auto& g : groups) {
        // time the kernel on this group's tiles only, for each shape; the
        // state is not advanced (same source buffer, step not incremented)
        float best = 1e30f;
        int best_s = saved[g.second[0]];
        for (int sidx = 0; sidx < flb::kNumShapes && !rc; ++sidx) {
            std::vector<int4> t;
            const int* sh = flb::kShapes[sidx];
            for (int r : g.second) {
                b->shape[r] = sidx;
                const HostModel& m = b->m[r];
                const int nx = (m.X + sh[0] - 1) / sh[0], ny = (m.Y + sh[1] - 1) / sh[1], nz = (m.Z + sh[2] - 1) / sh[2];
                for (int k = 0; k < nz; ++k)
                    for (int j = 0; j < ny; ++j)
                        for (int i = 0; i < nx; ++i) t.push_back(make_int4(r, i, j, k));
            }
            if ((rc = build_tiles(b))) break;  // parameters with the candidate shape
            int4* d_t = nullptr;
            cudaError_t e = cudaMalloc(&d_t, t.size() * sizeof(int4));
            if (e == cudaSuccess) e = cudaMemcpy(d_t, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice);
            float ms = 0.f;
            for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first launch warms up
                cudaEventRecord(e0, b->stream);
                for (int it = 0; it < 5; ++it) {
                    if (b->off32)
                        flb::k_step_batch<true>
                            <<<b->grid, 128, 0, b->stream>>>(b->args[b->cur], d_t, (int)t.size(), b->d_step);
                    else
                        flb::k_step_batch<false>
                            <<<b->grid, 128, 0, b->stream>>>(b->args[b->cur], d_t, (int)t.size(), b->d_step);
                }
                cudaEventRecord(e1, b->stream);
                e = cudaEventSynchronize(e1);
                float m1 = 0.f;
                cudaEventElapsedTime(&m1, e0, e1);
                if (rep > 0) ms += m1;
            }
            if (d_t) cudaFree(d_t);
            if (e != cudaSuccess) rc = bfail(FLB_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
            else if (ms < best) {
                best = ms;
                best_s = sidx;
            }
        }
        for (int r : g.second) b->shape[r] = best_s;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        b->shape = saved;
        build_tiles(b);
        return rc;
    }
    if ((rc = build_tiles(b))) return rc;
    if (shapes_out)
        for (int r = 0; r < b->n; ++r)
            for (int d = 0; d < 3; ++d) shapes_out[3 * r + d] = flb::kShapes[b->shape[r]][d];
    return FLB_OK;
}

int flb_batch_mode_variance(flb_batch* b, double* out)
{
    FLB_TRACE();
    if (!b || !out) return bfail(FLB_EINVAL, "NULL argument");
    Dev guard(b->device);
    const flb::PrecOps& ops = flb::ops_fp32();
    if (!b->partials) {
        int rows = 0;
        for (int r = 0; r < b->n; ++r) rows = std::max(rows, ops.partial_rows_max(b->m[r]));
        BCUDA(cudaMalloc(&b->partials, (size_t)rows * 38 * sizeof(double)));
        BCUDA(cudaMalloc(&b->red, (size_t)b->n * 38 * sizeof(double)));
    }
    b->mv_count += 1;
    // every replica's 38 column sums into its own row of red (the partial-sum
    // rows are reused in stream order), then one copy and one wait
    for (int r = 0; r < b->n; ++r) {
        int nrows = 0;
        BCUDA(ops.mode_partials(b->m[r], rep_src(b, r), b->partials, &nrows, b->stream));
        BCUDA(flb::sum_columns(b->partials, nrows, 38, b->red + 38 * (size_t)r, b->stream));
    }
    std::vector<double> h((size_t)b->n * 38);
    BCUDA(cudaMemcpyAsync(h.data(), b->red, h.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    for (int r = 0; r < b->n; ++r) {
        const double V = (double)b->m[r].V;
        for (int a = 0; a < 19; ++a) {
            const double mean = h[38 * r + a] / V;
            b->mv_sum[19 * r + a] += h[38 * r + 19 + a] / V - mean * mean;
            out[19 * r + a] = b->mv_sum[19 * r + a] / b->mv_count;
        }
    }
    return FLB_OK;
}

int flb_batch_structure_factor(flb_batch* b, int replica, double* S, int mode, int accumulate)
{
    FLB_TRACE();
    if (!b) return bfail(FLB_EINVAL, "batch is NULL");
    if (replica < 0 || replica >= b->n || mode < 0 || mode >= 19) return bfail(FLB_EINVAL, "replica or mode out of range");
    Dev guard(b->device);
    const flb::PrecOps& ops = flb::ops_fp32();
    const HostModel& m = b->m[replica];
    if (!b->fft) {
        long vmax = 0;
        for (auto& mm : b->m) vmax = std::max(vmax, mm.V);
        BCUDA(cudaMalloc(&b->fft, vmax * sizeof(double2)));
        BCUDA(cudaMalloc(&b->fft_scratch, vmax * sizeof(double2)));
        BCUDA(cudaMalloc(&b->sk_tmp, vmax * sizeof(double)));
    }
    double* target = nullptr;
    if (accumulate) {
        auto& slot = b->sk_acc[{replica, mode}];
        if (!slot.first) BCUDA(cudaMalloc(&slot.first, m.V * sizeof(double)));
        if (slot.second == 0) BCUDA(cudaMemsetAsync(slot.first, 0, m.V * sizeof(double), b->stream));
        target = slot.first;
        slot.second += 1;
    }
    // FP32 states: FP32 transform, |F|^2 summed in FP64 (as flb_structure_factor)
    BCUDA(ops.mode_field(m, rep_src(b, replica), mode, b->fft, true, b->stream));
    BCUDA(flb::fft3d((float2*)b->fft, m.X, m.Y, m.Z, (float2*)b->fft_scratch, b->stream));
    BCUDA(flb::power_spectrum((const float2*)b->fft, m.V, target, b->sk_tmp, b->stream));
    if (S) {
        if (accumulate)
            BCUDA(flb::scale_copy(target, 1.0 / b->sk_acc[{replica, mode}].second, m.V, b->sk_tmp, b->stream));
        BCUDA(cudaMemcpyAsync(S, b->sk_tmp, m.V * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        BCUDA(cudaStreamSynchronize(b->stream));
    }
    return FLB_OK;
}

int flb_batch_get_populations(flb_batch* b, int replica, double* f)
{
    FLB_TRACE();
    if (!b || !f) return bfail(FLB_EINVAL, "NULL argument");
    if (replica < 0 || replica >= b->n) return bfail(FLB_EINVAL, "replica out of range");
    Dev guard(b->device);
    const HostModel& m = b->m[replica];
    double* d = nullptr;
    BCUDA(cudaMalloc(&d, 19 * m.V * sizeof(double)));
    cudaError_t e = flb::ops_fp32().get_pop(m, rep_src(b, replica), d, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, 19 * m.V * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(d);
    if (e != cudaSuccess) return bfail(FLB_ECUDA, std::string("flb_batch_get_populations: ") + cudaGetErrorString(e));
    return FLB_OK;
}

int flb_batch_info(flb_batch* b, int* n, long long* sites, uint64_t* step)
{
    if (!b) return bfail(FLB_EINVAL, "batch is NULL");
    if (n) *n = b->n;
    if (sites) *sites = b->sites;
    if (step) *step = b->step;
    return FLB_OK;
}

int flb_batch_synchronize(flb_batch* b)
{
    if (!b) return bfail(FLB_EINVAL, "batch is NULL");
    Dev guard(b->device);
    BCUDA(cudaStreamSynchronize(b->stream));
    return FLB_OK;
}

void flb_batch_destroy(flb_batch* b)
{
    if (!b) return;
    Dev guard(b->device);
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    void* ptrs[] = {b->buf[0], b->buf[1], b->d_step, b->tiles, b->partials, b->red, b->fft, b->fft_scratch, b->sk_tmp};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& kv : b->sk_acc)
        if (kv.second.first) cudaFree(kv.second.first);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

}  // extern "C"
