// flb_kernels.cuh -- kernel templates of the fluctuating LB step.
//
// Storage: two structure-of-arrays buffers of deviations g_i = f_i - w_i rho0,
// layout [i][z][y][x].  A buffer holds the post-collision populations f* of
// the last completed step; the paper's pre-collision state is recovered by a
// pull, f^LB_i(r, t) = f*_i(r - c_i, t - 1) (streaming of Eq. (lbe-gen)).
//
// One step (Sec. V, Eq. (lbe-mom)) per site r, fused in one kernel:
//   pull g_i(r - c_i) -> moments -> relax, force, noise -> back-transform
//   -> write g*_i(r) into the other buffer.
// The non-ideal fluid (App. A) first needs rho on a neighbourhood: the density
// gather kernel writes drho(r) = sum_i g*_i(r - c_i) for every site, and the
// step kernel stages drho of its tile plus a 2-site halo in shared memory,
// evaluates mu = psi'(rho) - kappa lap rho on the tile plus a 1-site halo and
// F = -rho grad mu at each site.
#pragma once

#include <type_traits>

#include "flb_device.cuh"

namespace flb {

// Indices of the 3x3x3 neighbourhood of (x, y, z) on a periodic X*Y*Z lattice:
// xv[1+dx] + rb[1+dy][1+dz] is the site index of (x+dx, y+dy, z+dz).
struct Nbhd {
    int xv[3];
    int rb[3][3];
    __device__ __forceinline__ Nbhd(int x, int y, int z, int X, int Y, int Z)
    {
        xv[0] = wrap_once(x - 1, X);
        xv[1] = x;
        xv[2] = wrap_once(x + 1, X);
        const int yv[3] = {wrap_once(y - 1, Y), y, wrap_once(y + 1, Y)};
        const int zv[3] = {wrap_once(z - 1, Z), z, wrap_once(z + 1, Z)};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) rb[a][b] = X * (yv[a] + Y * zv[b]);
    }
    // index of r - c for c = (cx, cy, cz)
    __device__ __forceinline__ int src(int cx, int cy, int cz) const { return xv[1 - cx] + rb[1 - cy][1 - cz]; }
};

// Velocity tables for the pull / scatter addressing (same order as the API).
template <class L>
struct Vel;
template <>
struct Vel<D2Q9> {
    __device__ __forceinline__ static int cx(int i)
    {
        return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
    }
    __device__ __forceinline__ static int cy(int i)
    {
        return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
    }
    __device__ __forceinline__ static int cz(int) { return 0; }
    __device__ __forceinline__ static double w(int i) { return i == 0 ? 4.0 / 9 : i < 5 ? 1.0 / 9 : 1.0 / 36; }
};
template <>
struct Vel<D3Q19> {
    __device__ __forceinline__ static int cx(int i)
    {
        return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
             : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
    }
    __device__ __forceinline__ static int cy(int i)
    {
        return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
             : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
    }
    __device__ __forceinline__ static int cz(int i)
    {
        return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
             : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
    }
    __device__ __forceinline__ static double w(int i) { return i == 0 ? 1.0 / 3 : i < 7 ? 1.0 / 18 : 1.0 / 36; }
};

// Pull g_i(r - c_i) for all i.
template <class L, class R, class S>
__device__ __forceinline__ void pull(const S* __restrict__ src, long V, const Nbhd& nb, R g[L::Q])
{
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
        g[i] = load_s<R>(src + (long)i * V + nb.src(Vel<L>::cx(i), Vel<L>::cy(i), Vel<L>::cz(i)));
}

// Base pointers of the Q population planes of the source and destination
// buffers (in the parameter bank): a population address is one 32-bit site
// offset from a per-direction base.
template <class S>
struct Planes {
    const S* src[19];
    S* dst[19];
};

template <class S>
Planes<S> make_planes(const void* src, void* dst, int Q, long V)
{
    Planes<S> p{};
    for (int i = 0; i < Q; ++i) {
        p.src[i] = (const S*)src + (long)i * V;
        p.dst[i] = (S*)dst + (long)i * V;
    }
    return p;
}

// Pull g_i(r - c_i) through the plane pointers (LAST: last read of these
// populations in this step).
template <class L, bool LAST, class R, class S>
__device__ __forceinline__ void pull_planes(const Planes<S>& P, const Nbhd& nb, R g[L::Q])
{
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const S* p = P.src[i] + nb.src(Vel<L>::cx(i), Vel<L>::cy(i), Vel<L>::cz(i));
        g[i] = LAST ? load_last<R>(p) : load_s<R>(p);
    }
}

// Cache-hinted FP32 loads (PTX ld.global with an L1 eviction priority and an
// L2 prefetch size).  stream2/stream1: populations read once per step by the
// ideal step -- not allocated in L1, the L2 fetches 256-byte sectors.
// keep4/keep1: the fused non-ideal step's density gather, whose lines the
// collision of the same tile pulls again two planes later -- kept in L1 with
// the evict_last priority, 256-byte L2 fetches.
__device__ __forceinline__ float2 ld_stream2(const float* p)
{
    float2 v;
    asm("ld.global.L1::no_allocate.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream1(const float* p)
{
    float v;
    asm("ld.global.L1::no_allocate.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float4 ld_keep4(const float* p)
{
    float4 v;
    asm("ld.global.L1::evict_last.L2::256B.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_keep1(const float* p)
{
    float v;
    asm("ld.global.L1::evict_last.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// Storage access of the two-sites-per-thread kernels, FP32 in registers:
// S = float, or __nv_bfloat16 (a bf16 widens to FP32 exactly by a 16-bit
// shift; stores round to nearest even, as store_s does).  stream: the ideal
// step's hints above; keep: the density gather's; plain: the collision's pull.
template <class S>
struct Packed;
template <>
struct Packed<float> {
    static __device__ __forceinline__ float2 stream2(const float* p) { return ld_stream2(p); }
    static __device__ __forceinline__ float stream1(const float* p) { return ld_stream1(p); }
    static __device__ __forceinline__ float4 keep4(const float* p) { return ld_keep4(p); }
    static __device__ __forceinline__ float keep1(const float* p) { return ld_keep1(p); }
    static __device__ __forceinline__ float2 plain2(const float* p) { return *reinterpret_cast<const float2*>(p); }
    static __device__ __forceinline__ float plain1(const float* p) { return *p; }
    static __device__ __forceinline__ void store2(float* p, float2 v) { __stcs(reinterpret_cast<float2*>(p), v); }
};
template <>
struct Packed<__nv_bfloat16> {
    using B = __nv_bfloat16;
    static __device__ __forceinline__ float lo(uint32_t u) { return __uint_as_float(u << 16); }
    static __device__ __forceinline__ float hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }
    static __device__ __forceinline__ float2 stream2(const B* p)
    {
        uint32_t u;
        asm("ld.global.L1::no_allocate.L2::256B.b32 %0, [%1];" : "=r"(u) : "l"(p));
        return make_float2(lo(u), hi(u));
    }
    static __device__ __forceinline__ float stream1(const B* p)
    {
        unsigned short u;
        asm("ld.global.L1::no_allocate.L2::256B.b16 %0, [%1];" : "=h"(u) : "l"(p));
        return lo(u);
    }
    static __device__ __forceinline__ float4 keep4(const B* p)
    {
        uint32_t a, b;
        asm("ld.global.L1::evict_last.L2::256B.v2.b32 {%0, %1}, [%2];" : "=r"(a), "=r"(b) : "l"(p));
        return make_float4(lo(a), hi(a), lo(b), hi(b));
    }
    static __device__ __forceinline__ float keep1(const B* p)
    {
        unsigned short u;
        asm("ld.global.L1::evict_last.L2::256B.b16 %0, [%1];" : "=h"(u) : "l"(p));
        return lo(u);
    }
    static __device__ __forceinline__ float2 plain2(const B* p)
    {
        const uint32_t u = *reinterpret_cast<const uint32_t*>(p);
        return make_float2(lo(u), hi(u));
    }
    static __device__ __forceinline__ float plain1(const B* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void store2(B* p, float2 v)
    {
        const __nv_bfloat162 b = __float22bfloat162_rn(v);
        __stcs(reinterpret_cast<unsigned int*>(p), *reinterpret_cast<const unsigned int*>(&b));
    }
};

// ---------------------------------------------------------------------------
// Step parameters
// ---------------------------------------------------------------------------
template <class R>
struct StepArgs {
    Coll<R> c;
    int X, Y, Z;
    long V;
    // non-ideal fluid: psi'(rho) = A (rho - rho_c) + B (rho - rho_c)^3, with
    // rho - rho_c = drho + rho0_minus_rhoc; mu = psi' - kappa lap rho.
    // pgrad = 1 when psi is the total bulk free energy: F = -rho grad mu gains
    // cs^2 grad rho = sum_i w_i c_i rho(r + c_i), which cancels the LB's own
    // ideal-gas pressure gradient (Eq. (he-force)); pgrad = 0 otherwise.
    R A, B, kappa, rho0_minus_rhoc, pgrad;
    int nzc;  // z-marching kernels: planes per block (the z extent of a block's column)
};

// ---------------------------------------------------------------------------
// Density gather: drho(r) = sum_i g*_i(r - c_i), the density deviation the
// coming step sees (needed on a neighbourhood by the force).
// ---------------------------------------------------------------------------
template <class L, class R, class S>
__global__ void k_density(const S* __restrict__ src, R* __restrict__ drho, int X, int Y, int Z)
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
    drho[x + (long)X * (y + (long)Y * z)] = m[0];
}

// ---------------------------------------------------------------------------
// Fused pull + collide (+ force) + store.  Block = TX*TY*TZ threads, one site
// each.  NONIDEAL adds the shared-memory mu / F stencils; their density tile
// (tile + 2-site halo) comes from the field drho, or with GATHER from the
// populations themselves (each halo site's pulls summed as k_density does),
// which saves the separate density launch and field.
// ---------------------------------------------------------------------------
template <class L, class R, class S, bool NONIDEAL, int TX, int TY, int TZ, bool GATHER = false>
__global__ void __launch_bounds__(TX* TY* TZ)
    k_step(const StepArgs<R> a, const __grid_constant__ Planes<S> P, const R* __restrict__ drho)
{
    constexpr int HZ = (L::D == 3) ? 2 : 0;      // halo of rho in z
    constexpr int RX = TX + 4, RY = TY + 4, RZ = TZ + 2 * HZ;
    constexpr int MX = TX + 2, MY = TY + 2, MZ = TZ + (HZ ? 2 : 0);
    constexpr int NT = TX * TY * TZ;
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    const int z = blockIdx.z * TZ + threadIdx.z;
    const int X = a.X, Y = a.Y, Z = a.Z;

    R F[3] = {R(0), R(0), R(0)};
    if constexpr (NONIDEAL) {
        __shared__ R srho[RZ * RY * RX];
        __shared__ R smu[MZ * MY * MX];
        const int tid = threadIdx.x + TX * (threadIdx.y + TY * threadIdx.z);
        const int x0 = blockIdx.x * TX - 2, y0 = blockIdx.y * TY - 2, z0 = blockIdx.z * TZ - HZ;
        for (int e = tid; e < RZ * RY * RX; e += NT) {
            const int lx = e % RX, ly = (e / RX) % RY, lz = e / (RX * RY);
            const int gx = wrap_any(x0 + lx, X), gy = wrap_any(y0 + ly, Y), gz = wrap_any(z0 + lz, Z);
            if constexpr (GATHER) {
                const Nbhd nh(gx, gy, gz, X, Y, Z);
                R g[L::Q], m[L::Q];
#pragma unroll
                for (int i = 0; i < L::Q; ++i)
                    g[i] = load_s<R>(P.src[i] + nh.src(Vel<L>::cx(i), Vel<L>::cy(i), Vel<L>::cz(i)));
                L::moments(g, m);
                srho[e] = m[0];
            } else {
                srho[e] = drho[gx + (long)X * (gy + (long)Y * gz)];
            }
        }
        __syncthreads();
        // mu = psi'(rho) - kappa lap rho on the tile + 1 halo;
        // lap phi = 6 sum_i w_i (phi(r + c_i) - phi(r))
        for (int e = tid; e < MZ * MY * MX; e += NT) {
            const int mx = e % MX, my = (e / MX) % MY, mz = e / (MX * MY);
            const int cidx = (mx + 1) + RX * ((my + 1) + RY * (mz + (HZ ? 1 : 0)));
            const R r0 = srho[cidx];
            R lap = R(0);
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                const int o = Vel<L>::cx(i) + RX * (Vel<L>::cy(i) + RY * Vel<L>::cz(i));
                lap += R(Vel<L>::w(i)) * (srho[cidx + o] - r0);
            }
            lap *= R(6);
            const R d = r0 + a.rho0_minus_rhoc;
            smu[e] = d * (a.A + a.B * d * d) - a.kappa * lap;
        }
        __syncthreads();
        // grad mu = 3 sum_i w_i c_i mu(r + c_i); F = -rho grad mu
        const int cm = (threadIdx.x + 1) + MX * ((threadIdx.y + 1) + MY * (threadIdx.z + (HZ ? 1 : 0)));
        R gx = R(0), gy = R(0), gz = R(0);
#pragma unroll
        for (int i = 1; i < L::Q; ++i) {
            const int o = Vel<L>::cx(i) + MX * (Vel<L>::cy(i) + MY * Vel<L>::cz(i));
            const R wm = R(Vel<L>::w(i)) * smu[cm + o];
            if (Vel<L>::cx(i)) gx += R(Vel<L>::cx(i)) * wm;
            if (Vel<L>::cy(i)) gy += R(Vel<L>::cy(i)) * wm;
            if (Vel<L>::cz(i)) gz += R(Vel<L>::cz(i)) * wm;
        }
        const int cr = (threadIdx.x + 2) + RX * ((threadIdx.y + 2) + RY * (threadIdx.z + HZ));
        const R rho = a.c.rho0 + srho[cr];
        const R pre = R(-3) * rho;
        F[0] = pre * gx;
        F[1] = pre * gy;
        F[2] = pre * gz;
        if (a.pgrad != R(0)) {
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                const R wr = R(Vel<L>::w(i)) * srho[cr + Vel<L>::cx(i) + RX * (Vel<L>::cy(i) + RY * Vel<L>::cz(i))];
                if (Vel<L>::cx(i)) F[0] += R(Vel<L>::cx(i)) * wr;
                if (Vel<L>::cy(i)) F[1] += R(Vel<L>::cy(i)) * wr;
                if (Vel<L>::cz(i)) F[2] += R(Vel<L>::cz(i)) * wr;
            }
        }
    }
    if (x >= X || y >= Y || z >= Z) return;
    const Nbhd nb(x, y, z, X, Y, Z);
    R g[L::Q];
    pull_planes<L, false>(P, nb, g);
    const int s = x + X * (y + Y * z);
    if constexpr (L::D == 3)
        L::template collide<NONIDEAL>(g, F[0], F[1], F[2], a.c, (uint32_t)s, a.c.step);
    else
        L::collide(g, F[0], F[1], a.c, (uint32_t)s, a.c.step);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) store_stream(P.dst[i] + s, g[i]);
}

// ---------------------------------------------------------------------------
// Modified-equilibrium model (Sec. IV.C), D2Q9: the pressure
// p = p0(rho) - kappa rho lap rho and the square-gradient stress enter the
// equilibrium (D2Q9::collide_swift); no force.  The density deviation comes
// from the gather kernel (tile + 1 halo in shared memory), the coloured e/eps
// noise from swift_noise: xi_e = Re(xi[s]) / V, xi_eps = -Im(xi[s]) / V.
// p0 = rho psi' - psi (+ rho cs^2 when psi is the excess free energy, pgrad = 0).
// ---------------------------------------------------------------------------
template <class R>
using NoiseField = typename std::conditional<std::is_same<R, double>::value, double2, float2>::type;

template <class R, class S, int TX, int TY>
__global__ void __launch_bounds__(TX* TY)
    k_step_swift(const StepArgs<R> a, const __grid_constant__ Planes<S> P, const R* __restrict__ drho,
                 const NoiseField<R>* __restrict__ xi)
{
    using L = D2Q9;
    constexpr int RX = TX + 2, RY = TY + 2;
    __shared__ R srho[RY * RX];
    const int X = a.X, Y = a.Y;
    const int tid = threadIdx.x + TX * threadIdx.y;
    const int x0 = blockIdx.x * TX - 1, y0 = blockIdx.y * TY - 1;
    for (int e = tid; e < RX * RY; e += TX * TY)
        srho[e] = drho[wrap_any(x0 + e % RX, X) + (long)X * wrap_any(y0 + e / RX, Y)];
    __syncthreads();
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
    if (x >= X || y >= Y) return;
    const int c = (threadIdx.x + 1) + RX * (threadIdx.y + 1);
    const R r0 = srho[c];
    R lap = R(0), gx = R(0), gy = R(0);
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        const R v = srho[c + Vel<L>::cx(i) + RX * Vel<L>::cy(i)];
        lap += R(Vel<L>::w(i)) * (v - r0);
        if (Vel<L>::cx(i)) gx += R(Vel<L>::cx(i) * Vel<L>::w(i)) * v;
        if (Vel<L>::cy(i)) gy += R(Vel<L>::cy(i) * Vel<L>::w(i)) * v;
    }
    lap *= R(6);
    gx *= R(3);
    gy *= R(3);
    const R rho = a.c.rho0 + r0;
    const R d = r0 + a.rho0_minus_rhoc;
    const R psi = d * d * (R(0.5) * a.A + R(0.25) * a.B * d * d);
    const R psip = d * (a.A + a.B * d * d);
    const R pex = rho * psip - psi - a.pgrad * rho * R(1.0 / 3.0) - a.kappa * rho * lap;
    const int s = x + X * y;
    R xe = R(0), xp = R(0);
    if (a.c.noise) {
        const NoiseField<R> v = xi[s];
        const double iv = 1.0 / (double)a.V;
        xe = R(v.x * iv);
        xp = R(-v.y * iv);
    }
    const Nbhd nb(x, y, 0, X, Y, 1);
    R g[L::Q];
    pull_planes<L, false>(P, nb, g);
    L::collide_swift(g, pex, gx, gy, a.kappa, xe, xp, a.c, (uint32_t)s, a.c.step);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) store_stream(P.dst[i] + s, g[i]);
}

// ---------------------------------------------------------------------------
// Ideal gas, FP32 or BF16 storage, two sites (x, x+1) per thread with packed
// FP32 arithmetic (F2).  X must be even: a thread's pair then never straddles a
// row and its populations at (x, x+1) are aligned to the pair's size.  Pulls along c_x = 0 are
// single 8-byte loads; along c_x = +-1 the pair comes from (x-1, x) or
// (x+1, x+2).  Block = TXT x TY x TZ threads covering 2 TXT x TY x TZ sites.
// ---------------------------------------------------------------------------
template <class L, class S, int TXT, int TY, int TZ, int MINB = 1>
__global__ void __launch_bounds__(TXT* TY* TZ, MINB)
    k_step2(const StepArgs<float> a, const __grid_constant__ Planes<S> P)
{
    using A = Packed<S>;
    const int x = 2 * (blockIdx.x * TXT + threadIdx.x);
    const int y = blockIdx.y * TY + threadIdx.y;
    const int z = blockIdx.z * TZ + threadIdx.z;
    const int X = a.X, Y = a.Y, Z = a.Z;
    if (x >= X || y >= Y || z >= Z) return;
    const int xm = x == 0 ? X - 1 : x - 1;  // x - 1
    const int x2 = x + 2 == X ? 0 : x + 2;  // x + 2
    const int yv[3] = {wrap_once(y - 1, Y), y, wrap_once(y + 1, Y)};
    const int zv[3] = {wrap_once(z - 1, Z), z, wrap_once(z + 1, Z)};
    int rb[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) rb[i][j] = X * (yv[i] + Y * zv[j]);
    F2 g[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const S* p = P.src[i] + rb[1 - Vel<L>::cy(i)][1 - Vel<L>::cz(i)];
        const int cx = Vel<L>::cx(i);
        if (cx == 0)
            g[i] = mk2(A::stream2(p + x));
        else if (cx > 0)
            g[i] = F2(A::stream1(p + xm), A::stream1(p + x));
        else
            g[i] = F2(A::stream1(p + x + 1), A::stream1(p + x2));
    }
    const int s = x + X * (y + Y * z);
    L::template collide<false>(g, F2(0.f), F2(0.f), F2(0.f), a.c, (uint32_t)s, a.c.step);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) A::store2(P.dst[i] + s, g[i].v);
}

// Density gather for site pairs (x, x+1), packed FP32; X even.
template <int TXT, int TY, int TZ>
__global__ void __launch_bounds__(TXT* TY* TZ)
    k_density2(const __grid_constant__ Planes<float> P, float* __restrict__ drho, int X, int Y, int Z)
{
    using L = D3Q19;
    const int x = 2 * (blockIdx.x * TXT + threadIdx.x);
    const int y = blockIdx.y * TY + threadIdx.y;
    const int z = blockIdx.z * TZ + threadIdx.z;
    if (x >= X || y >= Y || z >= Z) return;
    const int xm = x == 0 ? X - 1 : x - 1, x2 = x + 2 == X ? 0 : x + 2;
    const int yv[3] = {wrap_once(y - 1, Y), y, wrap_once(y + 1, Y)};
    const int zv[3] = {wrap_once(z - 1, Z), z, wrap_once(z + 1, Z)};
    F2 g[L::Q], m[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const float* p = P.src[i] + X * (yv[1 - Vel<L>::cy(i)] + Y * zv[1 - Vel<L>::cz(i)]);
        const int cx = Vel<L>::cx(i);
        if (cx == 0)
            g[i] = mk2(*reinterpret_cast<const float2*>(p + x));
        else if (cx > 0)
            g[i] = F2(p[xm], p[x]);
        else
            g[i] = F2(p[x + 1], p[x2]);
    }
    L::moments(g, m);
    *reinterpret_cast<float2*>(drho + x + X * (y + Y * z)) = m[0].v;
}

// ---------------------------------------------------------------------------
// D3Q19 non-ideal fluid with the density gather fused in: one block owns a
// TX x TY column of sites and marches over a.nzc planes in z.  Iteration k pulls
// drho of plane zb+k+2 on the tile + 2-site halo (the tile interior's pulled
// populations are re-read from L2 by the collision two planes later),
// evaluates mu of plane zb+k+1 on the tile + 1-site halo, and collides plane
// zb+k with F = -rho grad mu.  The first iterations (k < 0) only fill the
// rings of 5 density planes and 3 chemical-potential planes kept in shared
// memory; the density never goes to DRAM.  Each stage appears once in the
// loop body so that the kernel stays small in the instruction cache.
// ---------------------------------------------------------------------------
template <class R, class S, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX* TY, MINB)
    k_step_march(const StepArgs<R> a, const __grid_constant__ Planes<S> P)
{
    using L = D3Q19;
    constexpr int NT = TX * TY, RX = TX + 4, RY = TY + 4, RP = RX * RY, MX = TX + 2, MY = TY + 2, MP = MX * MY;
    constexpr int NRH = (RP + NT - 1) / NT;  // halo density sites per thread
    __shared__ R srho[5][RP];
    __shared__ R smu[3][MP];
    const int tid = threadIdx.x + TX * threadIdx.y;
    const int X = a.X, Y = a.Y, Z = a.Z;
    const int XY = X * Y;
    const int xb = blockIdx.x * TX, yb = blockIdx.y * TY, zb = blockIdx.z * a.nzc;
    const int nz = min(a.nzc, Z - zb);

    // In-plane neighbourhood of this thread's density sites (fixed over z):
    // x - 1, x, x + 1 and the row offsets X*(y - 1), X*y, X*(y + 1).
    int hx[NRH][3], hy[NRH][3];
#pragma unroll
    for (int h = 0; h < NRH; ++h) {
        const int e = min(tid + h * NT, RP - 1);
        const int gx = wrap_any(xb - 2 + e % RX, X), gy = wrap_any(yb - 2 + e / RX, Y);
        hx[h][0] = wrap_once(gx - 1, X);
        hx[h][1] = gx;
        hx[h][2] = wrap_once(gx + 1, X);
        hy[h][0] = X * wrap_once(gy - 1, Y);
        hy[h][1] = X * gy;
        hy[h][2] = X * wrap_once(gy + 1, Y);
    }

    // this thread's chemical-potential sites: centre offset in the density plane
    constexpr int NMU = (MP + NT - 1) / NT;
    int mc[NMU];
#pragma unroll
    for (int j = 0; j < NMU; ++j) {
        const int e = min(tid + j * NT, MP - 1);
        mc[j] = (e % MX + 1) + RX * (e / MX + 1);
    }

    const int x = xb + threadIdx.x, y = yb + threadIdx.y;
    const int cm = (threadIdx.x + 1) + MX * (threadIdx.y + 1);
    const int cr = (threadIdx.x + 2) + RX * (threadIdx.y + 2);
    // ring slots, advanced by one each iteration: plane zb+k+2 of the density
    // goes to slot (k+4) mod 5 = ra + 2, the collision reads density slot
    // ra = (k+2) mod 5 and chemical-potential slots (k, k+1, k+2) mod 3.
    int ra = 3;       // (k + 2) mod 5 at k = -4
    int mb = 2;       // k mod 3 at k = -4
    int zc = wrap_any(zb - 2, Z);  // density plane being gathered, wrapped
#pragma unroll 1
    for (int k = -4; k < nz; ++k) {
        const int ra1 = ra == 4 ? 0 : ra + 1, ra2 = ra1 == 4 ? 0 : ra1 + 1;
        const int mb1 = mb == 2 ? 0 : mb + 1, mb2 = mb1 == 2 ? 0 : mb1 + 1;
        // (1) density of plane zb+k+2 on the tile + 2 halo: drho = sum_i g*_i(r - c_i)
        {
            const int zo[3] = {XY * (zc == 0 ? Z - 1 : zc - 1), XY * zc, XY * (zc == Z - 1 ? 0 : zc + 1)};
            R* out = srho[ra2];
#pragma unroll
            for (int h = 0; h < NRH; ++h) {
                const int e = tid + h * NT;
                if (e < RP) {
                    R g[L::Q], m[L::Q];
#pragma unroll
                    for (int i = 0; i < L::Q; ++i)
                        g[i] = load_s<R>(P.src[i] + (hx[h][1 - Vel<L>::cx(i)] + hy[h][1 - Vel<L>::cy(i)] +
                                                     zo[1 - Vel<L>::cz(i)]));
                    L::moments(g, m);
                    out[e] = m[0];
                }
            }
        }
        __syncthreads();
        // (2) mu = psi'(rho) - kappa lap rho of plane zb+k+1 on the tile + 1 halo
        if (k >= -2) {
            const R* rm = srho[ra];
            const R* r0 = srho[ra1];
            const R* rp = srho[ra2];
            R* out = smu[mb2];
#pragma unroll
            for (int j = 0; j < NMU; ++j) {
                const int e = tid + j * NT;
                if (e < MP) {
                    const int c = mc[j];
                    const R rc = r0[c];
                    R lap = R(0);
#pragma unroll
                    for (int i = 1; i < L::Q; ++i) {
                        const int cz = Vel<L>::cz(i);
                        const R* pl = cz > 0 ? rp : (cz < 0 ? rm : r0);
                        lap += R(Vel<L>::w(i)) * (pl[c + Vel<L>::cx(i) + RX * Vel<L>::cy(i)] - rc);
                    }
                    lap *= R(6);
                    const R d = rc + a.rho0_minus_rhoc;
                    out[e] = d * (a.A + a.B * d * d) - a.kappa * lap;
                }
            }
        }
        __syncthreads();
        // (3) collide plane zb+k with F = -rho grad mu, grad = 3 sum_i w_i c_i mu(r + c_i)
        if (k >= 0 && x < X && y < Y) {
            const int z = zb + k;
            const R* mlo = smu[mb];
            const R* mmid = smu[mb1];
            const R* mhi = smu[mb2];
            R gx = R(0), gy = R(0), gz = R(0);
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                const int cz = Vel<L>::cz(i);
                const R* pl = cz > 0 ? mhi : (cz < 0 ? mlo : mmid);
                const R wm = R(Vel<L>::w(i)) * pl[cm + Vel<L>::cx(i) + MX * Vel<L>::cy(i)];
                if (Vel<L>::cx(i)) gx += R(Vel<L>::cx(i)) * wm;
                if (Vel<L>::cy(i)) gy += R(Vel<L>::cy(i)) * wm;
                if (Vel<L>::cz(i)) gz += R(Vel<L>::cz(i)) * wm;
            }
            const R pre = R(-3) * (a.c.rho0 + srho[ra][cr]);
            R fx = pre * gx, fy = pre * gy, fz = pre * gz;
            if (a.pgrad != R(0)) {
                // + cs^2 grad rho from the density planes z-1, z, z+1
                const R* qlo = srho[ra == 0 ? 4 : ra - 1];
                const R* qmid = srho[ra];
                const R* qhi = srho[ra1];
#pragma unroll
                for (int i = 1; i < L::Q; ++i) {
                    const int cz = Vel<L>::cz(i);
                    const R* pl = cz > 0 ? qhi : (cz < 0 ? qlo : qmid);
                    const R wr = R(Vel<L>::w(i)) * pl[cr + Vel<L>::cx(i) + RX * Vel<L>::cy(i)];
                    if (Vel<L>::cx(i)) fx += R(Vel<L>::cx(i)) * wr;
                    if (Vel<L>::cy(i)) fy += R(Vel<L>::cy(i)) * wr;
                    if (Vel<L>::cz(i)) fz += R(Vel<L>::cz(i)) * wr;
                }
            }
            const Nbhd nb(x, y, z, X, Y, Z);
            R g[L::Q];
            pull_planes<L, true>(P, nb, g);
            const int s = x + X * (y + Y * z);
            L::collide(g, fx, fy, fz, a.c, (uint32_t)s, a.c.step);
#pragma unroll
            for (int i = 0; i < L::Q; ++i) store_stream(P.dst[i] + s, g[i]);
        }
        ra = ra1;
        mb = mb1;
        zc = zc == Z - 1 ? 0 : zc + 1;
    }
}


// ---------------------------------------------------------------------------
// Packed-FP32 form of k_step_march (FP32 or BF16 storage S): each thread owns
// the two sites (x, x+1) of its column pair, and every stage (density gather,
// mu, F, collision) works on site pairs with FADD2/FMUL2/FFMA2.  X must be
// even.  Same algorithm and ring layout as k_step_march; the density and mu
// planes are stored as float2 pairs.  GX = 4 (X % 4 == 0): the density gather
// works on quads of sites, one 4-element load per direction plus one
// 1-element load for c_x = +-1, and the density plane starts at x = xb - 4 so
// that its quads stay aligned; GX = 2: it works on pairs and starts at
// xb - 2.  Excess free energy only (pgrad = 0): the total-free-energy force
// runs through k_step_march.
// ---------------------------------------------------------------------------
// SUMS: the block also adds up the mass deviation and the momentum of the
// state it steps from -- sum_i g_i and sum_i c_i g_i of each collided site's
// pulled populations, the first moments its collision forms -- and writes
// them as one row of 4 doubles (rows[block * 4 + 0..3]; FP32 within a warp,
// FP64 above).
template <class S, int TXT, int TY, int MINB, int GX, bool SUMS = false>
__global__ void __launch_bounds__(TXT* TY, MINB)
    k_step_march2(const StepArgs<float> a, const __grid_constant__ Planes<S> P, double* __restrict__ rows)
{
    using A = Packed<S>;
    F2 sum_r(0.f), sum_jx(0.f), sum_jy(0.f), sum_jz(0.f);
    using L = D3Q19;
    constexpr bool QUAD = GX == 4;
    constexpr int NT = TXT * TY;
    constexpr int OX = QUAD ? 4 : 2;                           // density plane starts at x = xb - OX
    constexpr int RY = TY + 4;                                 // density rows (tile + 2 halo)
    constexpr int RX = 2 * TXT + 2 * OX;                       // density floats per row
    constexpr int RXG = RX / GX, RPG = RXG * RY;               // gather items (pairs or quads) per plane
    constexpr int MXP = TXT + 1, MY = TY + 2, MPP = MXP * MY;  // mu pairs per plane (tile + 1 halo)
    constexpr int MX = 2 * MXP;                                // mu floats per row
    __shared__ __align__(16) float srho[5][RX * RY];
    __shared__ __align__(16) float smu[3][MPP * 2];
    const int tid = threadIdx.x + TXT * threadIdx.y;
    const int X = a.X, Y = a.Y, Z = a.Z;
    const int XY = X * Y;
    const int xb = blockIdx.x * 2 * TXT, yb = blockIdx.y * TY, zb = blockIdx.z * a.nzc;
    const int nz = min(a.nzc, Z - zb);
    const bool small = X < RX || Y < RY;

    // gather items of this thread (first site gx, a multiple of GX): the sites
    // gx - 1, gx and gx + GX after periodic wrap, and the rows gy - 1, gy, gy + 1
    constexpr int NRH = (RPG + NT - 1) / NT;
    int hx[NRH][3], hy[NRH][3];
#pragma unroll
    for (int h = 0; h < NRH; ++h) {
        const int e = min(tid + h * NT, RPG - 1);
        const int gx0 = xb - OX + GX * (e % RXG), gy0 = yb - 2 + e / RXG;
        const int gx = small ? wrap_any(gx0, X) : wrap_once(gx0, X);
        const int gy = small ? wrap_any(gy0, Y) : wrap_once(gy0, Y);
        hx[h][0] = gx == 0 ? X - 1 : gx - 1;
        hx[h][1] = gx;
        hx[h][2] = gx + GX == X ? 0 : gx + GX;
        hy[h][0] = X * wrap_once(gy - 1, Y);
        hy[h][1] = X * gy;
        hy[h][2] = X * wrap_once(gy + 1, Y);
    }
    constexpr int NMU = (MPP + NT - 1) / NT;
    int mc[NMU];  // float offset of the first site of a mu pair in the density plane
#pragma unroll
    for (int j = 0; j < NMU; ++j) {
        const int e = min(tid + j * NT, MPP - 1);
        mc[j] = 2 * (e % MXP) + OX - 1 + RX * (e / MXP + 1);
    }

    const int x = xb + 2 * threadIdx.x, y = yb + threadIdx.y;
    const int cm = 2 * threadIdx.x + 1 + MX * (threadIdx.y + 1);   // first site in the mu plane
    const int cr = 2 * threadIdx.x + OX + RX * (threadIdx.y + 2);  // first site in the density plane
    int ra = 3, mb = 2;
    int zc = wrap_any(zb - 2, Z);
#pragma unroll 1
    for (int k = -4; k < nz; ++k) {
        const int ra1 = ra == 4 ? 0 : ra + 1, ra2 = ra1 == 4 ? 0 : ra1 + 1;
        const int mb1 = mb == 2 ? 0 : mb + 1, mb2 = mb1 == 2 ? 0 : mb1 + 1;
        // (1) density of plane zb+k+2, tile + 2 halo
        {
            const int zo[3] = {XY * (zc == 0 ? Z - 1 : zc - 1), XY * zc, XY * (zc == Z - 1 ? 0 : zc + 1)};
            float* out = srho[ra2];
#pragma unroll
            for (int h = 0; h < NRH; ++h) {
                const int e = tid + h * NT;
                if (e < RPG) {
                    if constexpr (QUAD) {
                        // sites gx .. gx+3: pulls from gx-1 .. gx+4
                        F2 glo[L::Q], ghi[L::Q], m[L::Q];
#pragma unroll
                        for (int i = 0; i < L::Q; ++i) {
                            const S* p = P.src[i] + hy[h][1 - Vel<L>::cy(i)] + zo[1 - Vel<L>::cz(i)];
                            const float4 v = A::keep4(p + hx[h][1]);
                            const int cx = Vel<L>::cx(i);
                            if (cx == 0) {
                                glo[i] = F2(v.x, v.y);
                                ghi[i] = F2(v.z, v.w);
                            } else if (cx > 0) {
                                glo[i] = F2(A::keep1(p + hx[h][0]), v.x);
                                ghi[i] = F2(v.y, v.z);
                            } else {
                                glo[i] = F2(v.y, v.z);
                                ghi[i] = F2(v.w, A::keep1(p + hx[h][2]));
                            }
                        }
                        L::moments(glo, m);
                        const float2 lo = m[0].v;
                        L::moments(ghi, m);
                        *reinterpret_cast<float4*>(out + 4 * e) = make_float4(lo.x, lo.y, m[0].v.x, m[0].v.y);
                    } else {
                        // sites gx, gx+1: pulls from gx-1 .. gx+2
                        F2 g[L::Q], m[L::Q];
#pragma unroll
                        for (int i = 0; i < L::Q; ++i) {
                            const S* p = P.src[i] + hy[h][1 - Vel<L>::cy(i)] + zo[1 - Vel<L>::cz(i)];
                            const int cx = Vel<L>::cx(i);
                            if (cx == 0)
                                g[i] = mk2(A::plain2(p + hx[h][1]));
                            else if (cx > 0)
                                g[i] = F2(A::plain1(p + hx[h][0]), A::plain1(p + hx[h][1]));
                            else
                                g[i] = F2(A::plain1(p + hx[h][1] + 1), A::plain1(p + hx[h][2]));
                        }
                        L::moments(g, m);
                        *reinterpret_cast<float2*>(out + 2 * e) = m[0].v;
                    }
                }
            }
        }
        __syncthreads();
        // (2) mu pairs of plane zb+k+1, tile + 1 halo
        if (k >= -2) {
            const float* rm = srho[ra];
            const float* r0 = srho[ra1];
            const float* rp = srho[ra2];
            float* out = smu[mb2];
#pragma unroll
            for (int j = 0; j < NMU; ++j) {
                const int e = tid + j * NT;
                if (e < MPP) {
                    const int c = mc[j];
                    const F2 rc = F2(r0[c], r0[c + 1]);
                    // sum_i w_i (rho_i - rho) = (1/18) (axis sum) + (1/36) (edge sum) - (2/3) rho
                    // (the Laplacian is 6 times it)
                    F2 sax(0.f), sed(0.f);
#pragma unroll
                    for (int i = 1; i < L::Q; ++i) {
                        const int cz = Vel<L>::cz(i);
                        const float* pl = cz > 0 ? rp : (cz < 0 ? rm : r0);
                        // c is odd: pairs at c + cx are aligned only for cx = +-1
                        const int o = c + Vel<L>::cx(i) + RX * Vel<L>::cy(i);
                        const F2 v = Vel<L>::cx(i) != 0 ? mk2(*reinterpret_cast<const float2*>(pl + o))
                                                        : F2(pl[o], pl[o + 1]);
                        if (i < 7)
                            sax += v;
                        else
                            sed += v;
                    }
                    const F2 lap = (1.0f / 18.0f) * sax + (1.0f / 36.0f) * sed - (2.0f / 3.0f) * rc;
                    const F2 d = rc + a.rho0_minus_rhoc;
                    const F2 mu = d * (a.A + a.B * (d * d)) - (6.0f * a.kappa) * lap;
                    out[2 * e] = mu.v.x;
                    out[2 * e + 1] = mu.v.y;
                }
            }
        }
        __syncthreads();
        // (3) collide the pair of plane zb+k with F = -rho grad mu
        if (k >= 0 && x < X && y < Y) {
            const int z = zb + k;
            const float* mlo = smu[mb];
            const float* mmid = smu[mb1];
            const float* mhi = smu[mb2];
            // sum_i w_i c_i mu_i (grad mu / 3; F = -3 rho times it) from the
            // differences mu(c) - mu(-c) of the nine velocity pairs (2p-1, 2p):
            // axis pairs weigh 1/18, edge pairs 1/36
            F2 dp[10];
#pragma unroll
            for (int q = 1; q <= 9; ++q) {
                F2 v2[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int i = 2 * q - 1 + h;
                    const int cz = Vel<L>::cz(i);
                    const float* pl = cz > 0 ? mhi : (cz < 0 ? mlo : mmid);
                    const int o = cm + Vel<L>::cx(i) + MX * Vel<L>::cy(i);
                    v2[h] = Vel<L>::cx(i) != 0 ? mk2(*reinterpret_cast<const float2*>(pl + o)) : F2(pl[o], pl[o + 1]);
                }
                dp[q] = v2[0] - v2[1];
            }
            // pairs 4..9: (1,1,0) (1,-1,0) (1,0,1) (1,0,-1) (0,1,1) (0,1,-1)
            const F2 gx = (1.0f / 18.0f) * dp[1] + (1.0f / 36.0f) * ((dp[4] + dp[5]) + (dp[6] + dp[7]));
            const F2 gy = (1.0f / 18.0f) * dp[2] + (1.0f / 36.0f) * ((dp[4] - dp[5]) + (dp[8] + dp[9]));
            const F2 gz = (1.0f / 18.0f) * dp[3] + (1.0f / 36.0f) * ((dp[6] - dp[7]) + (dp[8] - dp[9]));
            const F2 rho = a.c.rho0 + mk2(*reinterpret_cast<const float2*>(srho[ra] + cr));
            const F2 pre = -3.0f * rho;
            // pull the pair (its lines were fetched by the gather of this plane;
            // plain loads: measured faster than the last-use or evict-first hints)
            const int xm = x == 0 ? X - 1 : x - 1, x2 = x + 2 == X ? 0 : x + 2;
            const int yv[3] = {wrap_once(y - 1, Y), y, wrap_once(y + 1, Y)};
            const int zv[3] = {XY * wrap_once(z - 1, Z), XY * z, XY * wrap_once(z + 1, Z)};
            F2 g[L::Q];
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const S* p = P.src[i] + X * yv[1 - Vel<L>::cy(i)] + zv[1 - Vel<L>::cz(i)];
                const int cx = Vel<L>::cx(i);
                if (cx == 0)
                    g[i] = mk2(A::plain2(p + x));
                else if (cx > 0)
                    g[i] = F2(A::plain1(p + xm), A::plain1(p + x));
                else
                    g[i] = F2(A::plain1(p + x + 1), A::plain1(p + x2));
            }
            const int s = x + X * y + XY * z;
            if constexpr (SUMS) {
                // the pre-collision mass deviation and momentum the collision forms
                F2 first[4];
                L::collide(g, pre * gx, pre * gy, pre * gz, a.c, (uint32_t)s, a.c.step, first);
                sum_r += first[0];
                sum_jx += first[1];
                sum_jy += first[2];
                sum_jz += first[3];
            } else {
                L::collide(g, pre * gx, pre * gy, pre * gz, a.c, (uint32_t)s, a.c.step);
            }
#pragma unroll
            for (int i = 0; i < L::Q; ++i) A::store2(P.dst[i] + s, g[i].v);
        }
        ra = ra1;
        mb = mb1;
        zc = zc == Z - 1 ? 0 : zc + 1;
    }
    if constexpr (SUMS) {
        __shared__ double red[NT / 32][4];
        float v[4] = {sum_r.v.x + sum_r.v.y, sum_jx.v.x + sum_jx.v.y, sum_jy.v.x + sum_jy.v.y,
                      sum_jz.v.x + sum_jz.v.y};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        if ((tid & 31) == 0)
            for (int k = 0; k < 4; ++k) red[tid >> 5][k] = (double)v[k];
        __syncthreads();
        if (tid < 4) {
            double acc = 0.0;
            for (int w = 0; w < NT / 32; ++w) acc += red[w][tid];
            rows[4 * (blockIdx.x + (long)gridDim.x * (blockIdx.y + (long)gridDim.y * blockIdx.z)) + tid] = acc;
        }
    }
}

}  // namespace flb
