// flb_prec.cuh -- kernels and launchers instantiated once per (compute type R,
// storage type S): the fused step, the density gather, initial state,
// population exchange, observables and reduction partials.  Included by
// flb_fp64.cu, flb_fp32.cu and flb_bf16.cu only.
#pragma once

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "flb_internal.h"
#include "flb_kernels.cuh"

#ifndef FLB_MARCH_MINB
#define FLB_MARCH_MINB 3
#endif
#ifndef FLB_MARCH_TY
#define FLB_MARCH_TY 8
#endif
#ifndef FLB_PACKED
#define FLB_PACKED 1
#endif
#ifndef FLB_STEP2_TXT
#define FLB_STEP2_TXT 32
#endif
#ifndef FLB_STEP2_TY
#define FLB_STEP2_TY 2
#endif
#ifndef FLB_STEP2_TZ
#define FLB_STEP2_TZ 2
#endif
// Ideal-gas two-site step, minimum resident blocks per SM: 5 with FP32
// storage (96 registers, 48 bytes spilled, 20 warps per SM: measured faster
// than 4 blocks at 126 registers), 4 with BF16 storage (5 measured slower).
#ifndef FLB_STEP2_MINB
#define FLB_STEP2_MINB 5
#endif
#ifndef FLB_STEP2_MINB_BF16
#define FLB_STEP2_MINB_BF16 4
#endif
#ifndef FLB_MARCH2_MINB
#define FLB_MARCH2_MINB 3
#endif
#ifndef FLB_MARCH2_TY
#define FLB_MARCH2_TY 8
#endif

namespace flb {

// ---------------------------------------------------------------------------
// Host -> kernel parameters
// ---------------------------------------------------------------------------
template <class L, class R>
Coll<R> make_coll(const HostModel& m, uint64_t step)
{
    Coll<R> c{};
    c.rho0 = R(m.rho0);
    // Eq. (lbe-mom) per non-conserved mode a = D + 1 + k, divided by N_a:
    // relaxation omega_a / N_a, forcing prefactor (1 - omega_a / 2) / N_a, and
    // Eq. (noise-lbe): variance rho kT (2 - w) w N_a / cs^2 added to m_a, so
    // the kernel adds ns * sqrt(rho) * z to m_a / N_a.
    const int nstress = L::D * (L::D + 1) / 2;
    for (int k = 0; k < L::NNC; ++k) {
        const int a = L::D + 1 + k;
        const double om = (k == 0) ? m.om_b : (k < nstress) ? m.om_s : m.om_g;
        const double Na = L::N(a);
        c.rel[k] = R(-om / Na);
        if (k < nstress) c.frc[k] = R((1.0 - 0.5 * om) / Na);
        c.ns[k] = R(std::sqrt(m.kT * (2.0 - om) * om * Na * 3.0) / Na);
    }
    c.sqrt_rho0 = R(std::sqrt(m.rho0));
    c.noise = m.kT > 0.0;
    c.noise_local = m.noise_local;
    c.key = philox_keys(m.seed);
    c.step = (uint32_t)step;
    c.replica = m.replica;
    return c;
}

template <class L, class R>
StepArgs<R> make_args(const HostModel& m, uint64_t step)
{
    StepArgs<R> a{};
    a.c = make_coll<L, R>(m, step);
    a.X = m.X;
    a.Y = m.Y;
    a.Z = m.Z;
    a.V = m.V;
    a.A = R(m.A);
    a.B = R(m.B);
    a.kappa = R(m.kappa);
    a.rho0_minus_rhoc = R(m.rho0 - m.rho_c);
    a.pgrad = R(m.nonideal && m.total ? 1 : 0);
    a.nzc = std::min(m.zchunk > 0 ? m.zchunk : kZChunkDefault, m.Z);
    return a;
}

inline dim3 grid_for(const HostModel& m, dim3 b)
{
    return dim3((m.X + b.x - 1) / b.x, (m.Y + b.y - 1) / b.y, (m.Z + b.z - 1) / b.z);
}

template <class L>
inline dim3 site_block()
{
    return L::D == 3 ? dim3(32, 4, 2) : dim3(32, 8, 1);
}

// ---------------------------------------------------------------------------
// Auxiliary kernels
// ---------------------------------------------------------------------------

// Initial state f^eq(rho, u) (+ thermal modes), written as post-collision data
// at r - c_i so that the next pull returns it at r.
template <class R>
struct ThermalAmp {
    R tn[19];  // sqrt(kT N_a / cs^2) / N_a per mode
};

template <class L, class R, class S>
__global__ void k_init(const StepArgs<R> a, S* __restrict__ dst, const double* __restrict__ rho_in,
                       const double* __restrict__ u_in, int thermal, const ThermalAmp<R> amp)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x >= a.X || y >= a.Y || z >= a.Z) return;
    const long V = a.V;
    const int s = x + a.X * (y + a.Y * z);
    const R rho = rho_in ? R(rho_in[s]) : a.c.rho0;
    const R drho = rho_in ? R(rho_in[s] - (double)a.c.rho0) : R(0);
    R u[3] = {R(0), R(0), R(0)};
    if (u_in)
        for (int d = 0; d < L::D; ++d) u[d] = R(u_in[d * V + s]);
    R m[L::Q], g[L::Q];
    L::eq_moments(drho, rho, u[0], u[1], u[2], m);
#pragma unroll
    for (int q = 0; q < L::Q; ++q) m[q] *= R(1.0 / L::N(q));
    if (thermal) {
        // Eqs. (G-ideal), (mu-ideal): every mode a gets variance rho kT N_a / cs^2
        const R sr = a.c.noise_local ? sqrt(rho) : a.c.sqrt_rho0;
        R zz[4 * L::NCALL_ALL];
#pragma unroll
        for (int b = 0; b < L::NCALL_ALL; ++b)
            normals4(a.c.key, (uint32_t)s, 0u, (uint32_t)b | (1u << 8), a.c.replica, zz + 4 * b);
#pragma unroll
        for (int q = 0; q < L::Q; ++q) m[q] += amp.tn[q] * sr * zz[q];
    }
    L::from_moments(m, g);
    const Nbhd nb(x, y, z, a.X, a.Y, a.Z);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
        store_s(dst + (long)i * V + nb.src(Vel<L>::cx(i), Vel<L>::cy(i), Vel<L>::cz(i)), g[i]);
}

template <class L, class R, class S>
__global__ void k_get_pop(const S* __restrict__ src, double* __restrict__ out, double rho0, int X, int Y, int Z)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x >= X || y >= Y || z >= Z) return;
    const long V = (long)X * Y * Z;
    const int s = x + X * (y + Y * z);
    const Nbhd nb(x, y, z, X, Y, Z);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
        out[(long)i * V + s] = Vel<L>::w(i) * rho0 +
                               (double)load_s<R>(src + (long)i * V + nb.src(Vel<L>::cx(i), Vel<L>::cy(i), Vel<L>::cz(i)));
}

// f_i(r_k) = w_i rho0 + g_i pulled from r_k - c_i, for a list of sites r_k.
template <class L, class R, class S>
__global__ void k_get_sites(const S* __restrict__ src, const long long* __restrict__ sites, int n,
                            double* __restrict__ out, double rho0, int X, int Y, int Z)
{
    const long V = (long)X * Y * Z;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const long s = sites[k];
        const int x = (int)(s % X), y = (int)((s / X) % Y), z = (int)(s / ((long)X * Y));
        const Nbhd nb(x, y, z, X, Y, Z);
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            out[(long)i * n + k] =
                Vel<L>::w(i) * rho0 +
                (double)load_s<R>(src + (long)i * V + nb.src(Vel<L>::cx(i), Vel<L>::cy(i), Vel<L>::cz(i)));
    }
}

template <class L, class R, class S>
__global__ void k_set_pop(const double* __restrict__ in, S* __restrict__ dst, double rho0, int X, int Y, int Z)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x >= X || y >= Y || z >= Z) return;
    const long V = (long)X * Y * Z;
    const int s = x + X * (y + Y * z);
    const Nbhd nb(x, y, z, X, Y, Z);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
        store_s(dst + (long)i * V + nb.src(Vel<L>::cx(i), Vel<L>::cy(i), Vel<L>::cz(i)),
                R(in[(long)i * V + s] - Vel<L>::w(i) * rho0));
}

// Pre-collision deviations in the storage type, [i][s] (pull of the stored
// post-collision buffer) and the inverse scatter.
template <class L, class S>
__global__ void k_pull_state(const S* __restrict__ src, S* __restrict__ out, int X, int Y, int Z)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x >= X || y >= Y || z >= Z) return;
    const long V = (long)X * Y * Z;
    const int s = x + X * (y + Y * z);
    const Nbhd nb(x, y, z, X, Y, Z);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
        out[(long)i * V + s] = src[(long)i * V + nb.src(Vel<L>::cx(i), Vel<L>::cy(i), Vel<L>::cz(i))];
}
template <class L, class S>
__global__ void k_push_state(const S* __restrict__ in, S* __restrict__ dst, int X, int Y, int Z)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x >= X || y >= Y || z >= Z) return;
    const long V = (long)X * Y * Z;
    const int s = x + X * (y + Y * z);
    const Nbhd nb(x, y, z, X, Y, Z);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
        dst[(long)i * V + nb.src(Vel<L>::cx(i), Vel<L>::cy(i), Vel<L>::cz(i))] = in[(long)i * V + s];
}

// which: 0 rho, 1 u = (j + F/2)/rho, 2 all moments (m_0 = rho).
template <class L, class R, class S>
__global__ void k_moments(const S* __restrict__ src, double* __restrict__ out, int which,
                          const R* __restrict__ F, double rho0, int X, int Y, int Z)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x >= X || y >= Y || z >= Z) return;
    const long V = (long)X * Y * Z;
    const int s = x + X * (y + Y * z);
    const Nbhd nb(x, y, z, X, Y, Z);
    R g[L::Q], m[L::Q];
    pull<L>(src, V, nb, g);
    L::moments(g, m);
    const double rho = rho0 + (double)m[0];
    if (which == 0) {
        out[s] = rho;
    } else if (which == 1) {
        for (int d = 0; d < L::D; ++d) {
            const double Fd = F ? (double)F[d * V + s] : 0.0;
            out[d * V + s] = ((double)m[1 + d] + 0.5 * Fd) / rho;
        }
    } else {
#pragma unroll
        for (int q = 0; q < L::Q; ++q) out[(long)q * V + s] = (q == 0) ? rho : (double)m[q];
    }
}

// mu = psi'(rho) - kappa lap rho and F = -rho grad mu on the whole lattice
// (global-memory stencils; used for observables, not in the time step).
template <class L, class R>
__global__ void k_mu(const StepArgs<R> a, const R* __restrict__ drho, R* __restrict__ mu)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x >= a.X || y >= a.Y || z >= a.Z) return;
    const int s = x + a.X * (y + a.Y * z);
    const Nbhd nb(x, y, z, a.X, a.Y, a.Z);
    const R r0 = drho[s];
    R lap = R(0);
#pragma unroll
    for (int i = 1; i < L::Q; ++i)
        lap += R(Vel<L>::w(i)) * (drho[nb.src(-Vel<L>::cx(i), -Vel<L>::cy(i), -Vel<L>::cz(i))] - r0);
    lap *= R(6);
    const R d = r0 + a.rho0_minus_rhoc;
    mu[s] = d * (a.A + a.B * d * d) - a.kappa * lap;
}

template <class L, class R>
__global__ void k_force(const StepArgs<R> a, const R* __restrict__ drho, const R* __restrict__ mu, R* __restrict__ F)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x >= a.X || y >= a.Y || z >= a.Z) return;
    const int s = x + a.X * (y + a.Y * z);
    const Nbhd nb(x, y, z, a.X, a.Y, a.Z);
    R gr[3] = {R(0), R(0), R(0)}, pr[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        const int q = nb.src(-Vel<L>::cx(i), -Vel<L>::cy(i), -Vel<L>::cz(i));  // r + c_i
        const R wm = R(Vel<L>::w(i)) * mu[q], wr = R(Vel<L>::w(i)) * drho[q];
        gr[0] += R(Vel<L>::cx(i)) * wm;
        gr[1] += R(Vel<L>::cy(i)) * wm;
        gr[2] += R(Vel<L>::cz(i)) * wm;
        pr[0] += R(Vel<L>::cx(i)) * wr;
        pr[1] += R(Vel<L>::cy(i)) * wr;
        pr[2] += R(Vel<L>::cz(i)) * wr;
    }
    const R pre = R(-3) * (a.c.rho0 + drho[s]);
    for (int d = 0; d < 3; ++d) F[d * a.V + s] = pre * gr[d] + a.pgrad * pr[d];
}

// Block sum of NV values per thread into out[0..NV) (one row per block): warp
// sums in the values' own type (32 terms; FP32 values stay off GB300's slow
// FP64 pipe), FP64 across the warps and, in k_sum_columns, across blocks.
template <int NV, class V>
__device__ __forceinline__ void block_sum_row(V v[NV], double* __restrict__ row)
{
    __shared__ double red[32][NV];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < NV; ++k) red[warp][k] = (double)v[k];
    __syncthreads();
    const int nw = (nthr + 31) / 32;
    for (int k = tid; k < NV; k += nthr) {
        double acc = 0.0;
        for (int w = 0; w < nw; ++w) acc += red[w][k];
        row[k] = acc;
    }
}

__device__ __forceinline__ long block_linear()
{
    return blockIdx.x + (long)gridDim.x * (blockIdx.y + (long)gridDim.y * blockIdx.z);
}

// Per block: sum m_a and sum m_a^2 of the pre-collision moments (m_0 = drho).
template <class L, class R, class S>
__global__ void k_mode_partials(const S* __restrict__ src, double* __restrict__ partials, int X, int Y, int Z)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    R v[2 * L::Q];
    for (int q = 0; q < 2 * L::Q; ++q) v[q] = R(0);
    if (x < X && y < Y && z < Z) {
        const long V = (long)X * Y * Z;
        const Nbhd nb(x, y, z, X, Y, Z);
        R g[L::Q], m[L::Q];
        pull<L>(src, V, nb, g);
        L::moments(g, m);
#pragma unroll
        for (int q = 0; q < L::Q; ++q) {
            v[q] = m[q];
            v[L::Q + q] = m[q] * m[q];
        }
    }
    block_sum_row<2 * L::Q>(v, partials + block_linear() * (2 * L::Q));
}

// Per block: sum of g and of g c over the stored buffer (a permutation of the
// pre-collision populations, so the totals are those of the state).
template <class L, class R, class S>
__global__ void k_cons_partials(const S* __restrict__ src, double* __restrict__ partials, int X, int Y, int Z)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (x < X && y < Y && z < Z) {
        const long V = (long)X * Y * Z;
        const int s = x + X * (y + Y * z);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const double gi = (double)load_s<R>(src + (long)i * V + s);
            v[0] += gi;
            v[1] += Vel<L>::cx(i) * gi;
            v[2] += Vel<L>::cy(i) * gi;
            v[3] += Vel<L>::cz(i) * gi;
        }
    }
    block_sum_row<4>(v, partials + block_linear() * 4);
}

// Single-precision state: the same sums without FP64 arithmetic per population
// (the FP64 rate of the part is a small fraction of its FP32 rate).  Each
// thread walks the sites with a fixed stride and adds every population into
// (hi, lo) single-precision pairs by Knuth's TwoSum, so the rounding error of
// each addition is kept in lo; the pairs become doubles only for the block sum.
// The grid depends on V alone, so the result is deterministic.
constexpr int kConsThreads = 256, kConsBlocksMax = 152 * 8;

__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float b)
{
    const float s = hi + b;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (b - bb);
    hi = s;
}

template <class L, class S>
__global__ void __launch_bounds__(kConsThreads) k_cons_partials_sp(const S* __restrict__ src,
                                                                   double* __restrict__ partials, long V)
{
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    for (long s = blockIdx.x * (long)kConsThreads + threadIdx.x; s < V; s += (long)gridDim.x * kConsThreads) {
        float g[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) g[i] = load_s<float>(src + (long)i * V + s);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            two_sum_add(hi[0], lo[0], g[i]);
            if (Vel<L>::cx(i) != 0) two_sum_add(hi[1], lo[1], Vel<L>::cx(i) > 0 ? g[i] : -g[i]);
            if (Vel<L>::cy(i) != 0) two_sum_add(hi[2], lo[2], Vel<L>::cy(i) > 0 ? g[i] : -g[i]);
            if (Vel<L>::cz(i) != 0) two_sum_add(hi[3], lo[3], Vel<L>::cz(i) > 0 ? g[i] : -g[i]);
        }
    }
    double v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (double)hi[k] + (double)lo[k];
    block_sum_row<4>(v, partials + (long)blockIdx.x * 4);
}

inline int cons_blocks(long V)
{
    return (int)std::min<long>((V + kConsThreads - 1) / kConsThreads, kConsBlocksMax);
}

template <class L, class R, class S, class T>
__global__ void k_mode_field(const S* __restrict__ src, int mode, T* __restrict__ out, int X, int Y, int Z)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x >= X || y >= Y || z >= Z) return;
    const long V = (long)X * Y * Z;
    const Nbhd nb(x, y, z, X, Y, Z);
    R g[L::Q], m[L::Q];
    pull<L>(src, V, nb, g);
    L::moments(g, m);
    R v = m[0];
#pragma unroll
    for (int q = 1; q < L::Q; ++q)
        if (q == mode) v = m[q];
    using E = decltype(T::x);
    out[x + X * (y + Y * z)] = T{E(v), E(0)};
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <class R, class S>
struct Prec {
    // FP32 arithmetic on FP32 or BF16 storage: the two-sites-per-thread kernels
    static constexpr bool kPackedStorage =
        std::is_same<R, float>::value && (std::is_same<S, float>::value || std::is_same<S, __nv_bfloat16>::value);
    template <class L>
    static cudaError_t density_l(const HostModel& m, const void* pop, void* drho, cudaStream_t st)
    {
        const dim3 b = site_block<L>();
        k_density<L, R, S><<<grid_for(m, b), b, 0, st>>>((const S*)pop, (R*)drho, m.X, m.Y, m.Z);
        return cudaGetLastError();
    }
    static cudaError_t density(const HostModel& m, const void* pop, void* drho, cudaStream_t st)
    {
        if constexpr (std::is_same<R, float>::value && std::is_same<S, float>::value) {
            if (m.Q == 19 && m.X % 2 == 0 && FLB_PACKED) {
                constexpr int TXT = 16, TY = 4, TZ = 2;
                const dim3 b(TXT, TY, TZ);
                const dim3 g((m.X / 2 + TXT - 1) / TXT, (m.Y + TY - 1) / TY, (m.Z + TZ - 1) / TZ);
                k_density2<TXT, TY, TZ><<<g, b, 0, st>>>(make_planes<S>(pop, nullptr, 19, m.V), (float*)drho, m.X,
                                                          m.Y, m.Z);
                return cudaGetLastError();
            }
        }
        return m.Q == 19 ? density_l<D3Q19>(m, pop, drho, st) : density_l<D2Q9>(m, pop, drho, st);
    }

    template <class L, bool NI, int TX, int TY, int TZ, bool GATHER = false>
    static cudaError_t step_t(const HostModel& m, uint64_t step, const void* src, void* dst, const void* drho,
                              cudaStream_t st)
    {
        const StepArgs<R> a = make_args<L, R>(m, step);
        const dim3 b(TX, TY, TZ);
        k_step<L, R, S, NI, TX, TY, TZ, GATHER><<<grid_for(m, b), b, 0, st>>>(
            a, make_planes<S>(src, dst, L::Q, m.V), (const R*)drho);
        return cudaGetLastError();
    }
    // The step; with rows (non-NULL) also the mass deviation and momentum of
    // the state it steps from, as *nrows rows of 4 partial sums, where the
    // step kernel provides them (cudaErrorNotSupported elsewhere, before any
    // launch).
    static cudaError_t step(const HostModel& m, uint64_t t, const void* src, void* dst, const void* drho,
                            cudaStream_t st)
    {
        return step_rows(m, t, src, dst, drho, nullptr, nullptr, st);
    }
    static cudaError_t step_rows(const HostModel& m, uint64_t t, const void* src, void* dst, const void* drho,
                                 double* rows, int* nrows, cudaStream_t st)
    {
        if (rows && !(kPackedStorage && m.Q == 19 && m.nonideal && m.X % 2 == 0 && FLB_PACKED && !m.total))
            return cudaErrorNotSupported;
        if (m.Q == 9 && m.nonideal && m.model == 1) {
            const StepArgs<R> a = make_args<D2Q9, R>(m, t);
            const dim3 b(32, 8, 1);
            k_step_swift<R, S, 32, 8><<<grid_for(m, b), b, 0, st>>>(a, make_planes<S>(src, dst, 9, m.V),
                                                                      (const R*)drho,
                                                                      (const NoiseField<R>*)m.swift_xi);
            return cudaGetLastError();
        }
        if (m.Q == 19) {
            if (m.nonideal) {
                if constexpr (kPackedStorage) {
                    if (m.X % 2 == 0 && FLB_PACKED && !m.total) {
                        constexpr int TXT = 16, TY = FLB_MARCH2_TY;
                        const StepArgs<R> a = make_args<D3Q19, R>(m, t);
                        const dim3 b(TXT, TY, 1);
                        const dim3 g((m.X + 2 * TXT - 1) / (2 * TXT), (m.Y + TY - 1) / TY,
                                     (m.Z + a.nzc - 1) / a.nzc);
                        // density gather by quads of sites when rows hold whole quads
                        const Planes<S> pl = make_planes<S>(src, dst, 19, m.V);
                        if (rows) *nrows = (int)(g.x * g.y * g.z);
                        if (m.X % 4 == 0) {
                            if (rows)
                                k_step_march2<S, TXT, TY, FLB_MARCH2_MINB, 4, true><<<g, b, 0, st>>>(a, pl, rows);
                            else
                                k_step_march2<S, TXT, TY, FLB_MARCH2_MINB, 4><<<g, b, 0, st>>>(a, pl, nullptr);
                        } else {
                            if (rows)
                                k_step_march2<S, TXT, TY, FLB_MARCH2_MINB, 2, true><<<g, b, 0, st>>>(a, pl, rows);
                            else
                                k_step_march2<S, TXT, TY, FLB_MARCH2_MINB, 2><<<g, b, 0, st>>>(a, pl, nullptr);
                        }
                        return cudaGetLastError();
                    }
                }
                constexpr int TX = 32, TY = FLB_MARCH_TY;
                const StepArgs<R> a = make_args<D3Q19, R>(m, t);
                const dim3 b(TX, TY, 1);
                const dim3 g((m.X + TX - 1) / TX, (m.Y + TY - 1) / TY, (m.Z + a.nzc - 1) / a.nzc);
                k_step_march<R, S, TX, TY, (sizeof(R) == 8 ? 1 : FLB_MARCH_MINB)>
                    <<<g, b, 0, st>>>(a, make_planes<S>(src, dst, 19, m.V));
                return cudaGetLastError();
            }
            if constexpr (kPackedStorage) {
                if (m.X % 2 == 0 && FLB_PACKED) {
                    constexpr int TXT = FLB_STEP2_TXT, TY = FLB_STEP2_TY, TZ = FLB_STEP2_TZ;
                    const StepArgs<R> a = make_args<D3Q19, R>(m, t);
                    const dim3 b(TXT, TY, TZ);
                    const dim3 g((m.X / 2 + TXT - 1) / TXT, (m.Y + TY - 1) / TY, (m.Z + TZ - 1) / TZ);
                    constexpr int MINB = sizeof(S) == 4 ? FLB_STEP2_MINB : FLB_STEP2_MINB_BF16;
                    k_step2<D3Q19, S, TXT, TY, TZ, MINB>
                        <<<g, b, 0, st>>>(a, make_planes<S>(src, dst, 19, m.V));
                    return cudaGetLastError();
                }
            }
            return step_t<D3Q19, false, 32, 4, 2>(m, t, src, dst, drho, st);
        }
        // force model: the density tile is gathered inside the step
        if (m.nonideal) return step_t<D2Q9, true, 32, 8, 1, true>(m, t, src, dst, drho, st);
        return step_t<D2Q9, false, 32, 8, 1>(m, t, src, dst, drho, st);
    }

    template <class L>
    static cudaError_t init_l(const HostModel& m, void* dst, const double* rho, const double* u, int thermal,
                              cudaStream_t st)
    {
        const StepArgs<R> a = make_args<L, R>(m, 0);
        ThermalAmp<R> amp{};
        for (int q = 0; q < L::Q; ++q) amp.tn[q] = R(std::sqrt(3.0 * m.kT / L::N(q)));
        const dim3 b = site_block<L>();
        k_init<L, R, S><<<grid_for(m, b), b, 0, st>>>(a, (S*)dst, rho, u, thermal, amp);
        return cudaGetLastError();
    }
    static cudaError_t init(const HostModel& m, void* dst, const double* rho, const double* u, int thermal,
                            cudaStream_t st)
    {
        return m.Q == 19 ? init_l<D3Q19>(m, dst, rho, u, thermal, st) : init_l<D2Q9>(m, dst, rho, u, thermal, st);
    }

    static cudaError_t get_pop(const HostModel& m, const void* src, double* out, cudaStream_t st)
    {
        if (m.Q == 19) {
            const dim3 b = site_block<D3Q19>();
            k_get_pop<D3Q19, R, S><<<grid_for(m, b), b, 0, st>>>((const S*)src, out, m.rho0, m.X, m.Y, m.Z);
        } else {
            const dim3 b = site_block<D2Q9>();
            k_get_pop<D2Q9, R, S><<<grid_for(m, b), b, 0, st>>>((const S*)src, out, m.rho0, m.X, m.Y, m.Z);
        }
        return cudaGetLastError();
    }
    static cudaError_t set_pop(const HostModel& m, const double* in, void* dst, cudaStream_t st)
    {
        if (m.Q == 19) {
            const dim3 b = site_block<D3Q19>();
            k_set_pop<D3Q19, R, S><<<grid_for(m, b), b, 0, st>>>(in, (S*)dst, m.rho0, m.X, m.Y, m.Z);
        } else {
            const dim3 b = site_block<D2Q9>();
            k_set_pop<D2Q9, R, S><<<grid_for(m, b), b, 0, st>>>(in, (S*)dst, m.rho0, m.X, m.Y, m.Z);
        }
        return cudaGetLastError();
    }
    static cudaError_t moments(const HostModel& m, const void* src, double* out, int which, const void* F,
                               cudaStream_t st)
    {
        if (m.Q == 19) {
            const dim3 b = site_block<D3Q19>();
            k_moments<D3Q19, R, S><<<grid_for(m, b), b, 0, st>>>((const S*)src, out, which, (const R*)F, m.rho0,
                                                                  m.X, m.Y, m.Z);
        } else {
            const dim3 b = site_block<D2Q9>();
            k_moments<D2Q9, R, S><<<grid_for(m, b), b, 0, st>>>((const S*)src, out, which, (const R*)F, m.rho0,
                                                                 m.X, m.Y, m.Z);
        }
        return cudaGetLastError();
    }
    template <class L>
    static cudaError_t mu_force_l(const HostModel& m, const void* drho, void* mu, void* F, cudaStream_t st)
    {
        const StepArgs<R> a = make_args<L, R>(m, 0);
        const dim3 b = site_block<L>();
        k_mu<L, R><<<grid_for(m, b), b, 0, st>>>(a, (const R*)drho, (R*)mu);
        k_force<L, R><<<grid_for(m, b), b, 0, st>>>(a, (const R*)drho, (const R*)mu, (R*)F);
        return cudaGetLastError();
    }
    static cudaError_t mu_force(const HostModel& m, const void* drho, void* mu, void* F, cudaStream_t st)
    {
        return m.Q == 19 ? mu_force_l<D3Q19>(m, drho, mu, F, st) : mu_force_l<D2Q9>(m, drho, mu, F, st);
    }
    // The D2Q9 non-ideal step reads a density field gathered beforehand; the
    // D3Q19 one gathers the density itself.
    // a density field written before the step: only the modified-equilibrium
    // step reads one (the force-model steps gather their density themselves)
    static int needs_density(const HostModel& m) { return m.nonideal && m.Q == 9 && m.model == 1 ? 1 : 0; }
    static int rows(const HostModel& m)
    {
        const dim3 b = m.Q == 19 ? site_block<D3Q19>() : site_block<D2Q9>();
        const dim3 g = grid_for(m, b);
        return (int)(g.x * g.y * g.z);
    }
    static cudaError_t mode_partials(const HostModel& m, const void* src, double* partials, int* nrows,
                                     cudaStream_t st)
    {
        *nrows = rows(m);
        if (m.Q == 19) {
            const dim3 b = site_block<D3Q19>();
            k_mode_partials<D3Q19, R, S><<<grid_for(m, b), b, 0, st>>>((const S*)src, partials, m.X, m.Y, m.Z);
        } else {
            const dim3 b = site_block<D2Q9>();
            k_mode_partials<D2Q9, R, S><<<grid_for(m, b), b, 0, st>>>((const S*)src, partials, m.X, m.Y, m.Z);
        }
        return cudaGetLastError();
    }
    static cudaError_t cons_partials(const HostModel& m, const void* src, double* partials, int* nrows,
                                     cudaStream_t st)
    {
        if constexpr (std::is_same<R, float>::value) {
            // at most rows(m): cons_blocks(V) <= ceil(V / 256) <= the site grid
            *nrows = cons_blocks(m.V);
            if (m.Q == 19)
                k_cons_partials_sp<D3Q19, S><<<*nrows, kConsThreads, 0, st>>>((const S*)src, partials, m.V);
            else
                k_cons_partials_sp<D2Q9, S><<<*nrows, kConsThreads, 0, st>>>((const S*)src, partials, m.V);
            return cudaGetLastError();
        }
        *nrows = rows(m);
        if (m.Q == 19) {
            const dim3 b = site_block<D3Q19>();
            k_cons_partials<D3Q19, R, S><<<grid_for(m, b), b, 0, st>>>((const S*)src, partials, m.X, m.Y, m.Z);
        } else {
            const dim3 b = site_block<D2Q9>();
            k_cons_partials<D2Q9, R, S><<<grid_for(m, b), b, 0, st>>>((const S*)src, partials, m.X, m.Y, m.Z);
        }
        return cudaGetLastError();
    }
    template <class T>
    static cudaError_t mode_field_t(const HostModel& m, const void* src, int mode, T* out, cudaStream_t st)
    {
        if (m.Q == 19) {
            const dim3 b = site_block<D3Q19>();
            k_mode_field<D3Q19, R, S, T><<<grid_for(m, b), b, 0, st>>>((const S*)src, mode, out, m.X, m.Y, m.Z);
        } else {
            const dim3 b = site_block<D2Q9>();
            k_mode_field<D2Q9, R, S, T><<<grid_for(m, b), b, 0, st>>>((const S*)src, mode, out, m.X, m.Y, m.Z);
        }
        return cudaGetLastError();
    }
    static cudaError_t mode_field(const HostModel& m, const void* src, int mode, void* out, bool fp32, cudaStream_t st)
    {
        return fp32 ? mode_field_t(m, src, mode, (float2*)out, st) : mode_field_t(m, src, mode, (double2*)out, st);
    }

    static cudaError_t pull_state(const HostModel& m, const void* src, void* out, cudaStream_t st)
    {
        if (m.Q == 19) {
            const dim3 b = site_block<D3Q19>();
            k_pull_state<D3Q19, S><<<grid_for(m, b), b, 0, st>>>((const S*)src, (S*)out, m.X, m.Y, m.Z);
        } else {
            const dim3 b = site_block<D2Q9>();
            k_pull_state<D2Q9, S><<<grid_for(m, b), b, 0, st>>>((const S*)src, (S*)out, m.X, m.Y, m.Z);
        }
        return cudaGetLastError();
    }
    static cudaError_t push_state(const HostModel& m, const void* in, void* dst, cudaStream_t st)
    {
        if (m.Q == 19) {
            const dim3 b = site_block<D3Q19>();
            k_push_state<D3Q19, S><<<grid_for(m, b), b, 0, st>>>((const S*)in, (S*)dst, m.X, m.Y, m.Z);
        } else {
            const dim3 b = site_block<D2Q9>();
            k_push_state<D2Q9, S><<<grid_for(m, b), b, 0, st>>>((const S*)in, (S*)dst, m.X, m.Y, m.Z);
        }
        return cudaGetLastError();
    }

    static cudaError_t get_sites(const HostModel& m, const void* src, const long long* sites, int n, double* out,
                                 cudaStream_t st)
    {
        if (n <= 0) return cudaSuccess;
        const int nb = std::min((n + 127) / 128, 152 * 4);
        if (m.Q == 19)
            k_get_sites<D3Q19, R, S><<<nb, 128, 0, st>>>((const S*)src, sites, n, out, m.rho0, m.X, m.Y, m.Z);
        else
            k_get_sites<D2Q9, R, S><<<nb, 128, 0, st>>>((const S*)src, sites, n, out, m.rho0, m.X, m.Y, m.Z);
        return cudaGetLastError();
    }

    static const PrecOps& ops()
    {
        static const PrecOps o = {(int)sizeof(S), (int)sizeof(R), density, step, init, get_pop, set_pop, moments,
                                  mu_force, mode_partials, cons_partials, mode_field, rows, needs_density,
                                  pull_state, push_state, get_sites, step_rows};
        return o;
    }
};

}  // namespace flb
