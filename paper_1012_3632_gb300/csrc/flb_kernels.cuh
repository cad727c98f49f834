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

// ---------------------------------------------------------------------------
// Step parameters
// ---------------------------------------------------------------------------
template <class R>
struct StepArgs {
    Coll<R> c;
    int X, Y, Z;
    long V;
    // non-ideal fluid: psi'(rho) = A (rho - rho_c) + B (rho - rho_c)^3, with
    // rho - rho_c = drho + rho0_minus_rhoc
    R A, B, kappa, rho0_minus_rhoc;
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
// each.  NONIDEAL adds the shared-memory mu / F stencils.
// ---------------------------------------------------------------------------
template <class L, class R, class S, bool NONIDEAL, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX* TY* TZ)
    k_step(const StepArgs<R> a, const S* __restrict__ src, S* __restrict__ dst, const R* __restrict__ drho)
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
            srho[e] = drho[gx + (long)X * (gy + (long)Y * gz)];
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
        const R rho = a.c.rho0 + srho[(threadIdx.x + 2) + RX * ((threadIdx.y + 2) + RY * (threadIdx.z + HZ))];
        const R pre = R(-3) * rho;
        F[0] = pre * gx;
        F[1] = pre * gy;
        F[2] = pre * gz;
    }
    if (x >= X || y >= Y || z >= Z) return;
    const long V = a.V;
    const Nbhd nb(x, y, z, X, Y, Z);
    R g[L::Q];
    pull<L>(src, V, nb, g);
    const int s = x + X * (y + Y * z);
    if constexpr (L::D == 3)
        L::collide(g, F[0], F[1], F[2], a.c, (uint32_t)s);
    else
        L::collide(g, F[0], F[1], a.c, (uint32_t)s);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) store_s(dst + (long)i * V + s, g[i]);
}

}  // namespace flb
