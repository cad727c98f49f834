// flb_fft.cu -- precision-independent kernels: deterministic column sums for
// the reductions, a mixed-radix (2, 3, 4, 5) Stockham FFT in double precision
// for the structure factors, and the power spectrum accumulation.
//
// Structure factor of mode a (Sec. IV, Eq. (g-correl); Sec. VI equilibration
// ratios): S_a(k) = |sum_r dm_a(r) exp(-i k.r)|^2 / V, accumulated in double.
#include <cmath>
#include <mutex>

#include "flb_internal.h"

namespace flb {

// ---------------------------------------------------------------------------
// Column sums (one block per column, fixed order: deterministic)
// ---------------------------------------------------------------------------
__global__ void k_sum_columns(const double* __restrict__ partials, int nrows, int ncol, double* __restrict__ out,
                              double add0)
{
    __shared__ double sh[256];
    const int c = blockIdx.x;
    double acc = 0.0;
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) acc += partials[(long)r * ncol + c];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = c == 0 ? sh[0] + add0 : sh[0];
}

cudaError_t sum_columns(const double* partials, int nrows, int ncol, double* out, cudaStream_t s, double add0)
{
    k_sum_columns<<<ncol, 256, 0, s>>>(partials, nrows, ncol, out, add0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FFT
// ---------------------------------------------------------------------------
struct FftPlan {
    int L;
    int nrad;
    int rad[32];
};

// Factor L into radices 4, 2, 3, 5; false if another prime remains.
static bool make_plan(int L, FftPlan& p)
{
    p.L = L;
    p.nrad = 0;
    int n = L;
    while (n % 4 == 0) {
        p.rad[p.nrad++] = 4;
        n /= 4;
    }
    while (n % 2 == 0) {
        p.rad[p.nrad++] = 2;
        n /= 2;
    }
    while (n % 3 == 0) {
        p.rad[p.nrad++] = 3;
        n /= 3;
    }
    while (n % 5 == 0) {
        p.rad[p.nrad++] = 5;
        n /= 5;
    }
    return n == 1 && p.nrad <= 32;
}

// Complex arithmetic on double2 (FP64 transforms) and float2 (FP32 transforms).
template <class T>
__device__ __forceinline__ T cmul(T a, T b)
{
    return T{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class T>
__device__ __forceinline__ T cadd(T a, T b)
{
    return T{a.x + b.x, a.y + b.y};
}
template <class T>
__device__ __forceinline__ T csub(T a, T b)
{
    return T{a.x - b.x, a.y - b.y};
}

// Line geometry: line (i0, i1) starts at i0*s_in + i1*s_out, elements es apart.
struct LineGeom {
    int L;
    long es, s_in, s_out;
    int n_in;
};

// One Stockham pass (Govindaraju et al., SC'08 formulation): butterfly j of
// radix R with Ns = product of the radices already applied reads in[j + r L/R],
// twiddles by exp(-2 pi i r (j mod Ns) / (Ns R)), applies the R-point DFT and
// writes out[(j / Ns) Ns R + (j mod Ns) + r Ns].  tw[m] = exp(-2 pi i m / L).
template <int R, class T>
__device__ __forceinline__ void butterfly(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ tw,
                                          int L, int Ns, int j)
{
    using E = decltype(T::x);
    const int stride = L / R;
    const int k = j % Ns;
    T v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[j + r * stride];
    if (Ns > 1) {
        const int step = k * (L / (Ns * R));  // exp(-2 pi i k / (Ns R)) = tw[step]
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[(r * step) % L]);
    }
    T y[R];
    if constexpr (R == 2) {
        y[0] = cadd(v[0], v[1]);
        y[1] = csub(v[0], v[1]);
    } else if constexpr (R == 4) {
        const T a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        const T c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        y[0] = cadd(a, c);
        y[2] = csub(a, c);
        y[1] = T{b.x + d.y, b.y - d.x};  // b - i d
        y[3] = T{b.x - d.y, b.y + d.x};  // b + i d
    } else if constexpr (R == 3) {
        const E h = E(0.86602540378443864676);  // sqrt(3)/2
        const T t = cadd(v[1], v[2]), u = csub(v[1], v[2]);
        y[0] = cadd(v[0], t);
        const T m = T{v[0].x - E(0.5) * t.x, v[0].y - E(0.5) * t.y};
        y[1] = T{m.x + h * u.y, m.y - h * u.x};  // m - i h u
        y[2] = T{m.x - h * u.y, m.y + h * u.x};  // m + i h u
    } else {  // R == 5: direct 5-point DFT, exp(-2 pi i m / 5) = tw[m L / 5]
        const int f = L / 5;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            T acc = v[0];
#pragma unroll
            for (int r = 1; r < 5; ++r) acc = cadd(acc, cmul(v[r], tw[((q * r) % 5) * f]));
            y[q] = acc;
        }
    }
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[base + r * Ns] = y[r];
}

// The same pass for a power-of-two line (radices 4 and 2 only): the index
// arithmetic by shifts and masks instead of integer division (lgL = log2 L,
// lgNs = log2 Ns), o = the line's first element, buffers padded by pad16.
// Shared-memory line buffers of the power-of-two path skip one element after
// every 16 (an 8- or 16-byte element spans 2 or 4 banks), which spreads the
// strided accesses of the early passes over the banks.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

template <int R, class T>
__device__ __forceinline__ void butterfly_p2(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ tw,
                                             int lgL, int lgNs, int j, int o)
{
    constexpr int lgR = R == 2 ? 1 : 2;
    const int stride = 1 << (lgL - lgR);
    const int k = j & ((1 << lgNs) - 1);
    T v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[pad16(o + j + r * stride)];
    if (lgNs > 0) {
        const int step = k << (lgL - lgNs - lgR);  // k L / (Ns R)
        const int mask = (1 << lgL) - 1;
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[(r * step) & mask]);
    }
    T y[R];
    if constexpr (R == 2) {
        y[0] = cadd(v[0], v[1]);
        y[1] = csub(v[0], v[1]);
    } else {
        const T a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        const T c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        y[0] = cadd(a, c);
        y[2] = csub(a, c);
        y[1] = T{b.x + d.y, b.y - d.x};  // b - i d
        y[3] = T{b.x - d.y, b.y + d.x};  // b + i d
    }
    const int base = o + ((j >> lgNs) << (lgNs + lgR)) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[pad16(base + (r << lgNs))] = y[r];
}

// Twiddle table tw[m] = exp(-2 pi i m / L), m < L, built by every block of
// k_fft_lines in shared memory.  FP32 transforms: one FP32 sincospi per entry.
// FP64 transforms: m = a S + b with S = ceil(sqrt(L)), tw[m] = coarse[a] *
// fine[b] with coarse[a] = exp(-2 pi i a S / L), fine[b] = exp(-2 pi i b / L):
// about 2 sqrt(L) FP64 sincospi per block instead of L (FP64 is slow on this
// part), each entry within a few ulp.  scratch: >= S + ceil(L / S) entries.
__device__ __forceinline__ void fill_twiddles(float2* tw, int L, float2*)
{
    for (int m = threadIdx.x; m < L; m += blockDim.x) {
        float s, c;
        sincospif(-2.0f * ((float)m / (float)L), &s, &c);
        tw[m] = make_float2(c, s);
    }
}
__device__ __forceinline__ void fill_twiddles(double2* tw, int L, double2* scratch)
{
    int S = 1;
    while (S * S < L) ++S;
    const int A = (L + S - 1) / S;
    for (int t = threadIdx.x; t < S + A; t += blockDim.x) {
        const int m = t < S ? t : (t - S) * S;
        double s, c;
        sincospi(-2.0 * (double)m / (double)L, &s, &c);
        scratch[t] = make_double2(c, s);
    }
    __syncthreads();
    for (int m = threadIdx.x; m < L; m += blockDim.x) tw[m] = cmul(scratch[S + m / S], scratch[m % S]);
    __syncthreads();
}

constexpr int kFftThreads = 256, kFftLoads = 4096 / kFftThreads;

template <class T>
__global__ void __launch_bounds__(kFftThreads) k_fft_lines(T* __restrict__ data, const FftPlan plan, const LineGeom g, int B)
{
    using E = decltype(T::x);
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int L = g.L;
    const int BLp = B * L + ((B * L) >> 4) + 1;  // a line buffer, room for the pad16 layout
    T* b0 = sm;
    T* b1 = sm + BLp;
    T* tw = sm + 2 * BLp;
    fill_twiddles(tw, L, b1);  // b1 is free until the first radix pass
    const int i0 = blockIdx.x * B;
    const long o1 = (long)blockIdx.y * g.s_out;
    const int nl = min(B, g.n_in - i0);
    const int tot = nl * L;
    // power-of-two lines (and line counts): shifts and masks for the indices
    const bool p2 = (L & (L - 1)) == 0, nl2 = (nl & (nl - 1)) == 0;
    const int lgL = __ffs(L) - 1, lgnl = __ffs(nl) - 1;
    // all of a thread's loads first (a block holds at most 4096 elements, so at
    // most kFftLoads per thread at 256 threads), then the shared-memory stores:
    // the loads are in flight together instead of one after another
    T vin[kFftLoads];
    int sidx[kFftLoads];
#pragma unroll
    for (int q = 0; q < kFftLoads; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < tot) {
            int l, j;
            if (g.es == 1) {
                l = p2 ? e >> lgL : e / L;
                j = p2 ? e & (L - 1) : e % L;
            } else {
                l = nl2 ? e & (nl - 1) : e % nl;
                j = nl2 ? e >> lgnl : e / nl;
            }
            sidx[q] = p2 ? pad16(l * L + j) : l * L + j;
            vin[q] = data[(long)(i0 + l) * g.s_in + o1 + (long)j * g.es];
        }
    }
#pragma unroll
    for (int q = 0; q < kFftLoads; ++q)
        if (threadIdx.x + q * blockDim.x < tot) b0[sidx[q]] = vin[q];
    __syncthreads();
    int Ns = 1;
    T* cur = b0;
    T* nxt = b1;
    if (p2) {
        int lgNs = 0;
        for (int p = 0; p < plan.nrad; ++p) {
            const int lgR = plan.rad[p] == 4 ? 2 : 1;
            const int lgper = lgL - lgR;
            for (int t = threadIdx.x; t < (nl << lgper); t += blockDim.x) {
                const int l = t >> lgper, j = t & ((1 << lgper) - 1);
                if (lgR == 2)
                    butterfly_p2<4>(cur, nxt, tw, lgL, lgNs, j, l << lgL);
                else
                    butterfly_p2<2>(cur, nxt, tw, lgL, lgNs, j, l << lgL);
            }
            __syncthreads();
            lgNs += lgR;
            T* tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
    }
    for (int p = 0; p < (p2 ? 0 : plan.nrad); ++p) {
        const int R = plan.rad[p];
        const int per = L / R;
        for (int t = threadIdx.x; t < nl * per; t += blockDim.x) {
            const int l = t / per, j = t % per;
            switch (R) {
            case 2: butterfly<2>(cur + l * L, nxt + l * L, tw, L, Ns, j); break;
            case 3: butterfly<3>(cur + l * L, nxt + l * L, tw, L, Ns, j); break;
            case 4: butterfly<4>(cur + l * L, nxt + l * L, tw, L, Ns, j); break;
            default: butterfly<5>(cur + l * L, nxt + l * L, tw, L, Ns, j); break;
            }
        }
        __syncthreads();
        Ns *= R;
        T* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
#pragma unroll
    for (int q = 0; q < kFftLoads; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < tot) {
            int l, j;
            if (g.es == 1) {
                l = p2 ? e >> lgL : e / L;
                j = p2 ? e & (L - 1) : e % L;
            } else {
                l = nl2 ? e & (nl - 1) : e % nl;
                j = nl2 ? e >> lgnl : e / nl;
            }
            data[(long)(i0 + l) * g.s_in + o1 + (long)j * g.es] = cur[p2 ? pad16(l * L + j) : l * L + j];
        }
    }
}

// Direct DFT for lengths with prime factors above 5 (small test lattices),
// accumulated in double.
template <class T>
__global__ void k_dft_lines_naive(const T* __restrict__ in, T* __restrict__ out, const LineGeom g, int n_out)
{
    using E = decltype(T::x);
    const long tot = (long)g.n_in * n_out * g.L;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
        const int k = (int)(e % g.L);
        const long line = e / g.L;
        const int i0 = (int)(line % g.n_in);
        const long i1 = line / g.n_in;
        const long base = i0 * g.s_in + i1 * g.s_out;
        double2 acc = make_double2(0.0, 0.0);
        for (int j = 0; j < g.L; ++j) {
            const int m = (int)(((long)j * k) % g.L);
            double s, c;
            sincospi(-2.0 * (double)m / (double)g.L, &s, &c);
            const T v = in[base + j * g.es];
            acc = cadd(acc, cmul(make_double2(v.x, v.y), make_double2(c, s)));
        }
        out[base + k * g.es] = T{E(acc.x), E(acc.y)};
    }
}

bool fft_length_in_place(int L)
{
    FftPlan p;
    return L == 1 || (L <= 4096 && make_plan(L, p));
}

// Opt k_fft_lines into the largest dynamic shared memory it uses (two line
// buffers of B L <= 8192 elements and a twiddle table of L <= 4096 elements),
// once per device.
template <class T>
static cudaError_t fft_smem_optin()
{
    constexpr int kMaxDev = 128;
    static bool done[kMaxDev] = {false};
    static std::mutex mtx;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mtx);
    if (!done[dev]) {
        e = cudaFuncSetAttribute(k_fft_lines<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((2 * (4096 + 256 + 1) + 4096) * sizeof(T)));
        if (e != cudaSuccess) return e;
        done[dev] = true;
    }
    return cudaSuccess;
}

template <class T>
static cudaError_t fft_axis(T* data, T* scratch, int L, long es, long s_in, int n_in, long s_out, int n_out, long V,
                            cudaStream_t s)
{
    if (L == 1) return cudaSuccess;
    FftPlan plan;
    const LineGeom g{L, es, s_in, s_out, n_in};
    if (L <= 4096 && make_plan(L, plan)) {
        const int B = L >= 2048 ? 1 : (2048 / L < 16 ? 2048 / L : 16);
        const size_t smem = (2ull * (B * L + ((B * L) >> 4) + 1) + L) * sizeof(T);
        cudaError_t e = fft_smem_optin<T>();
        if (e != cudaSuccess) return e;
        const dim3 grid((n_in + B - 1) / B, n_out);
        k_fft_lines<T><<<grid, kFftThreads, smem, s>>>(data, plan, g, B);
        return cudaGetLastError();
    }
    k_dft_lines_naive<T><<<1024, 256, 0, s>>>(data, scratch, g, n_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(data, scratch, V * sizeof(T), cudaMemcpyDeviceToDevice, s);
}

cudaError_t fft_rows(double2* data, int X, int n, double2* scratch, cudaStream_t s)
{
    return fft_axis(data, scratch, X, 1, X, n, (long)X * n, 1, (long)X * n, s);
}

template <class T>
static cudaError_t fft3d_t(T* data, int X, int Y, int Z, T* scratch, cudaStream_t s)
{
    const long V = (long)X * Y * Z;
    cudaError_t e;
    // x lines: inner index y, outer z
    if ((e = fft_axis(data, scratch, X, 1, X, Y, (long)X * Y, Z, V, s)) != cudaSuccess) return e;
    // y lines: inner x, outer z
    if ((e = fft_axis(data, scratch, Y, X, 1, X, (long)X * Y, Z, V, s)) != cudaSuccess) return e;
    // z lines: inner x, outer y
    return fft_axis(data, scratch, Z, (long)X * Y, 1, X, X, Y, V, s);
}

cudaError_t fft3d(double2* data, int X, int Y, int Z, double2* scratch, cudaStream_t s)
{
    return fft3d_t(data, X, Y, Z, scratch, s);
}

cudaError_t fft3d(float2* data, int X, int Y, int Z, float2* scratch, cudaStream_t s)
{
    return fft3d_t(data, X, Y, Z, scratch, s);
}

__global__ void k_power(const double2* __restrict__ d, long V, double* __restrict__ acc, double* __restrict__ out)
{
    for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < V; s += (long)gridDim.x * blockDim.x) {
        const double p = (s == 0) ? 0.0 : (d[s].x * d[s].x + d[s].y * d[s].y) / (double)V;
        if (acc)
            acc[s] += p;
        else
            out[s] = p;
    }
}

// |F(k)|^2 / V of a single-precision transform: the square in FP32, the
// accumulation over snapshots in FP64.
__global__ void k_power_sp(const float2* __restrict__ d, long V, double* __restrict__ acc, double* __restrict__ out)
{
    const float inv = 1.0f / (float)V;
    for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < V; s += (long)gridDim.x * blockDim.x) {
        const float2 v = d[s];
        const double p = (s == 0) ? 0.0 : (double)((v.x * v.x + v.y * v.y) * inv);
        if (acc)
            acc[s] += p;
        else
            out[s] = p;
    }
}

cudaError_t power_spectrum(const double2* data, long V, double* acc, double* out, cudaStream_t s)
{
    long nb = (V + 255) / 256;
    if (nb > 152 * 32) nb = 152 * 32;
    k_power<<<(unsigned)nb, 256, 0, s>>>(data, V, acc, out);
    return cudaGetLastError();
}

__global__ void k_scale_copy(const double* __restrict__ in, double a, long V, double* __restrict__ out)
{
    for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < V; s += (long)gridDim.x * blockDim.x)
        out[s] = a * in[s];
}

cudaError_t scale_copy(const double* in, double a, long V, double* out, cudaStream_t s)
{
    long nb = (V + 255) / 256;
    if (nb > 152 * 32) nb = 152 * 32;
    k_scale_copy<<<(unsigned)nb, 256, 0, s>>>(in, a, V, out);
    return cudaGetLastError();
}

cudaError_t power_spectrum(const float2* data, long V, double* acc, double* out, cudaStream_t s)
{
    long nb = (V + 255) / 256;
    if (nb > 152 * 32) nb = 152 * 32;
    k_power_sp<<<(unsigned)nb, 256, 0, s>>>(data, V, acc, out);
    return cudaGetLastError();
}

}  // namespace flb
