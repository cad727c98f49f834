// flb_ws.cuh -- warp-specialised form of the fused non-ideal D3Q19 step
// (force model, App. A; one step of Sec. V, Eq. (lbe-mom)).
//
// Same arithmetic, stencils and z-marching as k_step_march2 (the density of
// plane z+2 gathered by quads of sites, mu of plane z+1, the collision of
// plane z), with the stages on separate warps of one 384-thread block:
//   warps 0-3 (producer):  density of the tile + 2-site halo and mu of the
//                           tile + 1-site halo, running up to DL planes ahead;
//   warps 4-11 (consumer): F = -rho grad mu, pull, collision and store of a
//                           32 x 16 tile, one site pair per thread.
// The two roles meet in rings of DL + 2 density and mu planes in shared
// memory.  Named barriers (PTX bar.sync / bar.arrive with the block's thread
// count) hand planes over: FULL(j), producer -> consumer, says that mu of
// plane j+1 is written (the density of j was written two planes earlier);
// EMPTY(j), consumer -> producer, says that the consumers are done with plane
// j, whose density and mu-(j-1) slots the producer refills DL planes later.
// Both kinds cycle over DL barrier ids; the producer waits for EMPTY(j - DL)
// before its iteration j, so neither kind is re-armed before its previous use
// completed, and the consumers skip the EMPTY arrivals that no producer
// iteration waits for (every barrier is complete when the block exits).
// Barrier 1 orders the producer's own gather and mu stages.
//
// 12 warps at up to 168 registers fill one SM's register file: one block per
// SM.  The consumers never wait for the gather's DRAM latency as long as the
// producer keeps DL planes ahead; the producer's loads touch the lines that
// the consumers pull a few planes later (L1 evict_last, 256-byte L2 fetches).
// Requires X % 32 == 0 and Y % 16 == 0 (whole tiles: every thread of the
// block takes part in every barrier); Z is any length, periodic wrap included.
#pragma once

#include "flb_kernels.cuh"

namespace flb {

__device__ __forceinline__ void nbar_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void nbar_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

constexpr int kWsTileX = 32, kWsTileY = 16, kWsThreads = 384;

template <class S, int DL, int PF>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_step_ws(const StepArgs<float> a, const __grid_constant__ Planes<S> P)
{
    using A = Packed<S>;
    using L = D3Q19;
    constexpr int TXT = kWsTileX / 2, TY = kWsTileY;       // consumer: 16 pairs x 16 rows
    constexpr int NC = TXT * TY, NP = kWsThreads - NC, NB = kWsThreads;
    static_assert(NP == 128, "four producer warps");
    constexpr int R = DL + 2;                               // ring depth
    constexpr int OX = 4;                                   // density plane starts at x = xb - 4
    constexpr int RY = TY + 4, RX = 2 * TXT + 2 * OX;       // 20 rows of 40 floats
    constexpr int RXG = RX / 4, RPG = RXG * RY;             // 200 quads per plane
    constexpr int MXP = TXT + 1, MY = TY + 2, MPP = MXP * MY;  // 306 mu pairs per plane
    constexpr int MX = 2 * MXP;
    constexpr int FULL0 = 2, EMPTY0 = 2 + DL;               // barrier ids (0: __syncthreads, 1: producer)
    static_assert(DL >= 2 && EMPTY0 + DL <= 16, "named barrier ids");
    __shared__ __align__(16) float srho[R][RX * RY];
    __shared__ __align__(16) float smu[R][MPP * 2];
    const int X = a.X, Y = a.Y, Z = a.Z;
    const int XY = X * Y;
    const int xb = blockIdx.x * kWsTileX, yb = blockIdx.y * TY, zb = blockIdx.z * a.nzc;
    const int nz = min(a.nzc, Z - zb);
    auto slot = [](int p) { return (p + 2 * R) % R; };  // ring slot of plane zb+p (p >= -2)

    if (threadIdx.x < NP) {
        // ---------------- producer: density and mu planes ----------------
        const int tid = threadIdx.x;
        // gather items (quads of sites): first site gx (a multiple of 4) after
        // periodic wrap, its left and right neighbours, rows gy - 1, gy, gy + 1
        constexpr int NRH = (RPG + NP - 1) / NP;
        int hx[NRH][3], hy[NRH][3];
#pragma unroll
        for (int h = 0; h < NRH; ++h) {
            const int e = min(tid + h * NP, RPG - 1);
            const int gx = wrap_once(xb - OX + 4 * (e % RXG), X);
            const int gy = wrap_once(yb - 2 + e / RXG, Y);
            hx[h][0] = gx == 0 ? X - 1 : gx - 1;
            hx[h][1] = gx;
            hx[h][2] = gx + 4 == X ? 0 : gx + 4;
            hy[h][0] = X * wrap_once(gy - 1, Y);
            hy[h][1] = X * gy;
            hy[h][2] = X * wrap_once(gy + 1, Y);
        }
        constexpr int NMU = (MPP + NP - 1) / NP;
        int mc[NMU];  // float offset of the first site of a mu pair in the density plane
#pragma unroll
        for (int j = 0; j < NMU; ++j) {
            const int e = min(tid + j * NP, MPP - 1);
            mc[j] = 2 * (e % MXP) + OX - 1 + RX * (e / MXP + 1);
        }
        int zc = wrap_any(zb - 2, Z);  // z of the plane gathered in iteration j: zb + j + 2
#pragma unroll 1
        for (int j = -4; j < nz; ++j) {
            if (j >= DL) nbar_sync(EMPTY0 + (j - DL) % DL, NB);
            // (0) L2 prefetch of the tile's own lines that the gather of plane
            // zb+j+2+PF reads (one 32-site row segment per direction and row;
            // the halo rows and columns are the neighbouring tiles' own lines)
            if constexpr (PF > 0) {
                if (j + PF < nz) {
                    int zp = zc + PF;
                    while (zp >= Z) zp -= Z;
#pragma unroll
                    for (int q = 0; q < (19 * TY + NP - 1) / NP; ++q) {
                        const int e = tid + q * NP;
                        if (e < 19 * TY) {
                            const int i = e / TY, r = e % TY;
                            // c_z of direction i, two bits per direction (c_z + 1)
                            const int cz = (int)((0x20a0954955ull >> (2 * i)) & 3u) - 1;
                            const int zz = wrap_once(zp - cz, Z);
                            const S* ptr = P.src[i] + (long)XY * zz + X * (yb + r) + xb;
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
                        }
                    }
                }
            }
            // (1) density of plane zb+j+2, tile + 2 halo
            {
                const int zo[3] = {XY * (zc == 0 ? Z - 1 : zc - 1), XY * zc, XY * (zc == Z - 1 ? 0 : zc + 1)};
                float* out = srho[slot(j + 2)];
#pragma unroll
                for (int h = 0; h < NRH; ++h) {
                    const int e = tid + h * NP;
                    if (e < RPG) {
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
                    }
                }
            }
            nbar_sync(1, NP);
            // (2) mu pairs of plane zb+j+1, tile + 1 halo
            if (j >= -2) {
                const float* rm = srho[slot(j)];
                const float* r0 = srho[slot(j + 1)];
                const float* rp = srho[slot(j + 2)];
                float* out = smu[slot(j + 1)];
#pragma unroll
                for (int q = 0; q < NMU; ++q) {
                    const int e = tid + q * NP;
                    if (e < MPP) {
                        const int c = mc[q];
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
            if (j >= 0) nbar_arrive(FULL0 + j % DL, NB);
            zc = zc == Z - 1 ? 0 : zc + 1;
        }
    } else {
        // ---------------- consumers: force, pull, collide, store ----------------
        const int c = threadIdx.x - NP;
        const int px = c % TXT, py = c / TXT;
        const int x = xb + 2 * px, y = yb + py;
        const int cm = 2 * px + 1 + MX * (py + 1);   // first site in the mu plane
        const int cr = 2 * px + OX + RX * (py + 2);  // first site in the density plane
        const int xm = x == 0 ? X - 1 : x - 1, x2 = x + 2 == X ? 0 : x + 2;
        const int yv[3] = {wrap_once(y - 1, Y), y, wrap_once(y + 1, Y)};
#pragma unroll 1
        for (int j = 0; j < nz; ++j) {
            nbar_sync(FULL0 + j % DL, NB);
            const int z = zb + j;
            const float* mlo = smu[slot(j - 1)];
            const float* mmid = smu[slot(j)];
            const float* mhi = smu[slot(j + 1)];
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
            const F2 rho = a.c.rho0 + mk2(*reinterpret_cast<const float2*>(srho[slot(j)] + cr));
            const F2 pre = -3.0f * rho;
            // pull the pair (the producer touched its lines a few planes ago)
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
            // the consumers are done with the shared planes of j once F and rho are formed
            if (j + DL < nz) nbar_arrive(EMPTY0 + j % DL, NB);
            const int s = x + X * y + XY * z;
            L::collide(g, pre * gx, pre * gy, pre * gz, a.c, (uint32_t)s, a.c.step);
#pragma unroll
            for (int i = 0; i < L::Q; ++i) A::store2(P.dst[i] + s, g[i].v);
        }
    }
}

}  // namespace flb
