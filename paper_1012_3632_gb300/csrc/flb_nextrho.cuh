// flb_nextrho.cuh -- D3Q19 force-model step that also produces the density the
// next step needs.
//
// The force F = -rho grad mu (App. A, Eq. (he-force) with psi the excess free
// energy) at a site needs mu on its neighbourhood and so the density of the
// coming step, rho(r) = rho0 + sum_i g*_i(r - c_i), on the tile plus a 2-site
// halo.  Instead of gathering those 19 populations per halo site again from
// memory, each step adds up, while its post-collision populations are still on
// chip, what its own tile streams into every site -- the coming density, split
// by the tile it comes from -- and the next step reads one or a few numbers
// per site.
//
// Tiles are 32 x 8 sites in x-y; a block of 16 x 8 threads (two sites per
// thread, packed FP32) marches a column of z planes of its tile, as
// k_step_march2 does.  The split is fixed by the tiling, not by the column
// length, so results do not depend on it:
//
//   rho(r) - rho0 = ((P_T0(r) + P_Tx(r)) + P_Ty(r)) + P_Txy(r)
//
// over the tile T0 that holds r and, for sites on its edge, the neighbouring
// tiles in x, in y and across the corner whose sites stream into r (terms
// that do not apply are left out).  The part of one tile is
//
//   P_T(r) = (B_T(r) + S_T(r)) + A_T(r),
//
// with S_T, B_T, A_T the sums of g*_i(r - c_i) over the directions with
// c_z = 0, +1, -1 whose source r - c_i lies in T, added in ascending i (a
// source outside T adds an exact zero).
//
// Storage, FP32 ("parts" buffer of V + Z * ntiles * 84 floats):
//   part[z X Y + y X + x]            P_T0(r): the part of the site's own tile
//   part[V + (z ntiles + t) 84 + j]  P_t at the ring of 84 sites around tile t
//       j = 0..33:  y = -1, x = j - 1;    j = 34..67: y = 8, x = j - 35
//       j = 68..75: x = -1, y = j - 68;   j = 76..83: x = 32, y = j - 76
//   (x, y local to the tile, t = tx + ntx ty).
// A block writes the complete part of every plane inside its column.  At the
// column ends pieces come from the neighbouring columns: the block writes the
// bottom plane's S with its A kept apart, the top plane's B + S, and the A
// (B) piece it streams into the plane below (above) the column, the last
// three into a per-column array `ext`; k_rho_fixup then completes the two end
// planes of every column with the same order of additions.
#pragma once

#include <type_traits>

#include "flb_kernels.cuh"

namespace flb {
namespace nr {

constexpr int TW = 32, TH = 8;                  // tile, sites
constexpr int TXT = TW / 2;                     // threads per tile row
constexpr int NT = TXT * TH;                    // threads per block
constexpr int NRING = 84;                       // ring sites around a tile
constexpr int FX = TW + 4, FY = TH + 2;         // post-collision plane: tile + 2 columns / 1 row of zeros
constexpr int FP = FX * FY;
constexpr int OX = 2;                           // density plane starts at x = xb - 2
constexpr int RX = TW + 2 * OX, RY = TH + 4;    // density plane: tile + 2 halo
constexpr int RPAIRS = RX * RY / 2;             // site pairs per density plane (216)
constexpr int NRI = (RPAIRS + NT - 1) / NT;     // pairs per thread
constexpr int MXP = TXT + 1, MY = TH + 2, MPP = MXP * MY;  // mu pairs per plane (tile + 1 halo)
constexpr int MX = 2 * MXP;
constexpr int NMU = (MPP + NT - 1) / NT;

// Offset of g*_i at tile-local (x, y) in the post-collision plane (one slot
// per direction; a border of zeros 2 columns and 1 row wide).
__host__ __device__ constexpr int foff(int i, int x, int y) { return i * FP + (y + 1) * FX + (x + 2); }

// The parts of one tile at the sites (x0, x0 + 1), y (tile-local) of the
// plane its post-collision populations f came from: S for that plane, B for
// the plane above (c_z = +1), A for the plane below (c_z = -1).
__device__ __forceinline__ void own_pieces(const float* f, int x0, int y, F2& S, F2& B, F2& A)
{
    auto p2 = [&](int i, int x, int yy) { return mk2(*reinterpret_cast<const float2*>(f + foff(i, x, yy))); };
    auto p1 = [&](int i, int x, int yy) { return f[foff(i, x, yy)]; };
    S = p2(0, x0, y);
    S += F2(p1(1, x0 - 1, y), p1(1, x0, y));                 // ( 1, 0, 0) from x - 1
    S += F2(p1(2, x0 + 1, y), p1(2, x0 + 2, y));             // (-1, 0, 0) from x + 1
    S += p2(3, x0, y - 1);                                   // ( 0, 1, 0) from y - 1
    S += p2(4, x0, y + 1);                                   // ( 0,-1, 0) from y + 1
    S += F2(p1(7, x0 - 1, y - 1), p1(7, x0, y - 1));         // ( 1, 1, 0)
    S += F2(p1(8, x0 + 1, y + 1), p1(8, x0 + 2, y + 1));     // (-1,-1, 0)
    S += F2(p1(9, x0 - 1, y + 1), p1(9, x0, y + 1));         // ( 1,-1, 0)
    S += F2(p1(10, x0 + 1, y - 1), p1(10, x0 + 2, y - 1));   // (-1, 1, 0)
    B = p2(5, x0, y);
    B += F2(p1(11, x0 - 1, y), p1(11, x0, y));               // ( 1, 0, 1)
    B += F2(p1(14, x0 + 1, y), p1(14, x0 + 2, y));           // (-1, 0, 1)
    B += p2(15, x0, y - 1);                                  // ( 0, 1, 1)
    B += p2(18, x0, y + 1);                                  // ( 0,-1, 1)
    A = p2(6, x0, y);
    A += F2(p1(12, x0 + 1, y), p1(12, x0 + 2, y));           // (-1, 0,-1)
    A += F2(p1(13, x0 - 1, y), p1(13, x0, y));               // ( 1, 0,-1)
    A += p2(16, x0, y + 1);                                  // ( 0,-1,-1)
    A += p2(17, x0, y - 1);                                  // ( 0, 1,-1)
}

// Offsets in the post-collision plane of the sources that stream into ring
// site j: o[0..2] the c_z = 0 directions in ascending i, o[3] the c_z = +1
// direction, o[4] the c_z = -1 direction (zeros where the source lies outside
// the tile).
__device__ __forceinline__ void ring_sources(int j, int o[5])
{
    if (j < 34) {  // y = -1: directions with c_y = -1
        const int x = j - 1;
        o[0] = foff(4, x, 0), o[1] = foff(8, x + 1, 0), o[2] = foff(9, x - 1, 0);
        o[3] = foff(18, x, 0), o[4] = foff(16, x, 0);
    } else if (j < 68) {  // y = 8: c_y = +1
        const int x = j - 35;
        o[0] = foff(3, x, 7), o[1] = foff(7, x - 1, 7), o[2] = foff(10, x + 1, 7);
        o[3] = foff(15, x, 7), o[4] = foff(17, x, 7);
    } else if (j < 76) {  // x = -1: c_x = -1
        const int y = j - 68;
        o[0] = foff(2, 0, y), o[1] = foff(8, 0, y + 1), o[2] = foff(10, 0, y - 1);
        o[3] = foff(14, 0, y), o[4] = foff(12, 0, y);
    } else {  // x = 32: c_x = +1
        const int y = j - 76;
        o[0] = foff(1, 31, y), o[1] = foff(7, 31, y - 1), o[2] = foff(9, 31, y + 1);
        o[3] = foff(11, 31, y), o[4] = foff(13, 31, y);
    }
}
__device__ __forceinline__ void ring_pieces(const float* f, const int o[5], float& S, float& B, float& A)
{
    S = (f[o[0]] + f[o[1]]) + f[o[2]];
    B = f[o[3]];
    A = f[o[4]];
}

// Write the pair's 19 post-collision populations to the post-collision plane.
__device__ __forceinline__ void put_plane(float* f, const F2 g[19], int x0, int y)
{
#pragma unroll
    for (int i = 0; i < 19; ++i) *reinterpret_cast<float2*>(f + foff(i, x0, y)) = g[i].v;
}

// The value a population has once stored in S (BF16 storage rounds it).
template <class S>
__device__ __forceinline__ F2 as_stored(F2 v)
{
    if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        const __nv_bfloat162 b = __float22bfloat162_rn(v.v);
        return mk2(__bfloat1622float2(b));
    } else {
        return v;
    }
}

// Where the reader finds the parts of one site pair (gx, gx + 1), gx even, of
// the density plane: .x its own tile's part (offset in a plane's own-part
// array); .y the ring part of the tile beside it in x for the site on that
// tile edge, as 2 offset + site, or -1; .z the ring part of the tile beside
// it in y for site 0 (site 1: .z + 1), or -1; .w the ring part of the tile
// across the corner for the x-edge site, or -1 (offsets in a plane's ring array).
__device__ __forceinline__ int4 pair_parts(int gx, int gy, int X, int ntx, int nty)
{
    const int tx = gx / TW, ty = gy / TH, lx = gx % TW, ly = gy % TH;
    const int txm = tx == 0 ? ntx - 1 : tx - 1, txp = tx == ntx - 1 ? 0 : tx + 1;
    const int tym = ty == 0 ? nty - 1 : ty - 1, typ = ty == nty - 1 ? 0 : ty + 1;
    int hx = -1, hy = -1, hd = -1, xs = 0;
    int ntxn = tx;  // tile in x that streams into the x-edge site
    if (lx == 0) {  // site 0 on the left edge: the left tile's column x = 32
        ntxn = txm;
        hx = (txm + ntx * ty) * NRING + 76 + ly;
    } else if (lx == TW - 2) {  // site 1 (x = 31) on the right edge: the right tile's column x = -1
        ntxn = txp;
        hx = (txp + ntx * ty) * NRING + 68 + ly;
        xs = 1;
    }
    if (ly == 0) {  // the tile below streams into row y = 8 of its ring
        hy = (tx + ntx * tym) * NRING + 34 + lx + 1;
        if (hx >= 0) hd = (ntxn + ntx * tym) * NRING + 34 + (xs == 0 ? 33 : 0);
    } else if (ly == TH - 1) {  // the tile above streams into row y = -1 of its ring
        hy = (tx + ntx * typ) * NRING + lx + 1;
        if (hx >= 0) hd = (ntxn + ntx * typ) * NRING + (xs == 0 ? 33 : 0);
    }
    return make_int4(gx + X * gy, hx >= 0 ? 2 * hx + xs : -1, hy, hd);
}

// Density deviation of the coming step at the pair from the parts of one
// plane: own part, then the tile beside in x, in y, across the corner.
__device__ __forceinline__ float2 read_pair(const float* __restrict__ Dp, const float* __restrict__ Hp, int4 p)
{
    float2 v = *reinterpret_cast<const float2*>(Dp + p.x);
    if (p.y >= 0) {
        const int xs = p.y & 1;
        float& s = xs ? v.y : v.x;
        s += Hp[p.y >> 1];
        if (p.z >= 0) {
            float& o = xs ? v.x : v.y;
            s += Hp[p.z + xs];
            o += Hp[p.z + 1 - xs];
            if (p.w >= 0) s += Hp[p.w];
        }
    } else if (p.z >= 0) {
        v.x += Hp[p.z];
        v.y += Hp[p.z + 1];
    }
    return v;
}

// Fetch a line into L2 ahead of its use, kept with the evict_last priority.
__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(p));
}

// Asynchronous global -> shared copies (cp.async): the data lands in shared
// memory while the thread goes on; cp_async_wait makes the calling thread's
// own copies visible to it.
__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Parts of one density plane staged in shared memory: per density pair its
// own-tile parts and the up to four ring parts read_pair adds (x-edge, y-edge
// for site 0 and site 1, corner).
struct PartsStage {
    float2 d[RPAIRS];
    float h[RPAIRS][4];
};

// Issue the copies of plane (Dp, Hp) for the pairs of this thread.
__device__ __forceinline__ void stage_parts(PartsStage& st, const int4* tpp, const float* __restrict__ Dp,
                                            const float* __restrict__ Hp, int tid)
{
#pragma unroll
    for (int h = 0; h < NRI; ++h) {
        const int e = tid + h * NT;
        if (e < RPAIRS) {
            const int4 p = tpp[e];
            cp_async8(&st.d[e], Dp + p.x);
            if (p.y >= 0) cp_async4(&st.h[e][0], Hp + (p.y >> 1));
            if (p.z >= 0) {
                cp_async4(&st.h[e][1], Hp + p.z);
                cp_async4(&st.h[e][2], Hp + p.z + 1);
            }
            if (p.w >= 0) cp_async4(&st.h[e][3], Hp + p.w);
        }
    }
    cp_async_commit();
}

// The density pair from staged parts: the same additions in the same order as read_pair.
__device__ __forceinline__ float2 staged_pair(const PartsStage& st, int e, int4 p)
{
    float2 v = st.d[e];
    if (p.y >= 0) {
        const int xs = p.y & 1;
        float& s = xs ? v.y : v.x;
        s += st.h[e][0];
        if (p.z >= 0) {
            float& o = xs ? v.x : v.y;
            s += st.h[e][1 + xs];
            o += st.h[e][2 - xs];
            if (p.w >= 0) s += st.h[e][3];
        }
    } else if (p.z >= 0) {
        v.x += st.h[e][1];
        v.y += st.h[e][2];
    }
    return v;
}

// Dynamic shared memory of k_step_nextrho: the post-collision plane and two
// staged parts planes.
constexpr size_t kDynSmem = 19 * FP * sizeof(float) + 2 * sizeof(PartsStage);

}  // namespace nr

// Arguments of the density parts (device pointers, FP32).
struct RhoParts {
    const float* in;   // complete parts of the state the step starts from
    float* out;        // parts of the state the step produces
    float* ext;        // column-end pieces: [3 ncol][XY + ntiles 84], kinds 0 = A below, 1 = B above, 2 = A of the bottom plane
    int ntx, nty;      // tiles per row and column
};


// ---------------------------------------------------------------------------
// The step.  Iteration k of a block's column (planes zb .. zb + nz - 1):
// (1) density of plane zb+k+2 on the tile + 2 halo from the parts the previous
// step wrote (and an L2 prefetch of the parts of plane zb+k+3); (2) the parts
// of the coming density that plane zb+k-1 streams, from the post-collision
// plane the last iteration left in shared memory, and mu of plane zb+k+1 on
// the tile + 1 halo; (3) an L2 prefetch of the populations the collision of
// plane zb+k+2 will pull, then the collision of plane zb+k with
// F = -rho grad mu, its store, and its post-collision plane.  SUMS: per-block
// mass and momentum sums of the state stepped from, as k_step_march2.
// ---------------------------------------------------------------------------
template <class S, int MINB, bool SUMS = false>
__global__ void __launch_bounds__(nr::NT, MINB)
    k_step_nextrho(const StepArgs<float> a, const __grid_constant__ Planes<S> P, const RhoParts rp,
                   double* __restrict__ rows)
{
    using namespace nr;
    using L = D3Q19;
    using Acc = Packed<S>;
    __shared__ __align__(16) float srho[5][RX * RY];
    __shared__ __align__(16) float smu[3][MPP * 2];
    __shared__ int4 tpp[RPAIRS];      // where each density pair's parts are
    __shared__ int tro[5][NRING];     // sources of each ring site
    extern __shared__ __align__(16) float dyn[];
    float* fpl = dyn;                                               // post-collision plane
    PartsStage* stg = reinterpret_cast<PartsStage*>(dyn + 19 * FP);  // staged parts, two planes
    F2 sum_r(0.f), sum_jx(0.f), sum_jy(0.f), sum_jz(0.f);
    const int tid = threadIdx.x + TXT * threadIdx.y;
    const int X = a.X, Y = a.Y, Z = a.Z;
    const int XY = X * Y;
    const long V = a.V;
    const int ntiles = rp.ntx * rp.nty;
    const int tile = blockIdx.x + rp.ntx * blockIdx.y;
    const int xb = blockIdx.x * TW, yb = blockIdx.y * TH, zb = blockIdx.z * a.nzc;
    const int nz = min(a.nzc, Z - zb);
    const int col = blockIdx.z;
    const long exs = (long)XY + (long)ntiles * NRING;  // elements of one ext plane
    const long ring_plane = (long)ntiles * NRING;

    for (int e = tid; e < 19 * FP; e += NT) fpl[e] = 0.f;
    for (int e = tid; e < RPAIRS; e += NT) {
        const int gx = wrap_once(xb - OX + 2 * (e % (RX / 2)), X), gy = wrap_any(yb - 2 + e / (RX / 2), Y);
        tpp[e] = pair_parts(gx, gy, X, rp.ntx, rp.nty);
    }
    if (tid < NRING) {
        int o[5];
        ring_sources(tid, o);
#pragma unroll
        for (int q = 0; q < 5; ++q) tro[q][tid] = o[q];
    }

    const int lx0 = 2 * threadIdx.x, ly = threadIdx.y;
    const int x = xb + lx0, y = yb + ly;
    const int xm = x == 0 ? X - 1 : x - 1, x2 = x + 2 == X ? 0 : x + 2;
    const int cm = lx0 + 1 + MX * (ly + 1);     // first site in the mu plane
    const int cr = lx0 + OX + RX * (ly + 2);    // first site in the density plane
    const int own = x + X * y;                  // site offset within a plane
    F2 acc1(0.f), acc2(0.f);  // own pair: B of plane s+1, B + S of plane s
    float racc1 = 0.f, racc2 = 0.f;

    // the parts of the coming density that plane zb + ks streams (post-collision
    // plane in fpl); ks = 0 and 1 and the top plane leave pieces for k_rho_fixup
    auto scatter = [&](int ks) {
        F2 pS, pB, pA;
        own_pieces(fpl, lx0, ly, pS, pB, pA);
        float rS = 0.f, rB = 0.f, rA = 0.f;
        if (tid < NRING) {
            const int o[5] = {tro[0][tid], tro[1][tid], tro[2][tid], tro[3][tid], tro[4][tid]};
            ring_pieces(fpl, o, rS, rB, rA);
        }
        const long rng = V + (long)tile * NRING + tid;
        if (ks == 0) {
            // A of the plane below the column (kind 0); S starts the bottom plane
            float* e0 = rp.ext + (3L * col + 0) * exs;
            *reinterpret_cast<float2*>(e0 + own) = pA.v;
            if (tid < NRING) e0[XY + (long)tile * NRING + tid] = rA;
            acc2 = pS;
            racc2 = rS;
        } else {
            const int zt = zb + ks - 1;
            if (ks == 1) {
                // bottom plane: its S as it is, its A apart (kind 2)
                float* e2 = rp.ext + (3L * col + 2) * exs;
                *reinterpret_cast<float2*>(e2 + own) = pA.v;
                if (tid < NRING) e2[XY + (long)tile * NRING + tid] = rA;
                *reinterpret_cast<float2*>(rp.out + (long)zt * XY + own) = acc2.v;
                if (tid < NRING) rp.out[rng + (long)zt * ring_plane] = racc2;
            } else {
                *reinterpret_cast<float2*>(rp.out + (long)zt * XY + own) = (acc2 + pA).v;
                if (tid < NRING) rp.out[rng + (long)zt * ring_plane] = racc2 + rA;
            }
            acc2 = acc1 + pS;
            racc2 = racc1 + rS;
        }
        acc1 = pB;
        racc1 = rB;
    };

    int ra = 3, mb = 2;
    int zc = wrap_any(zb - 2, Z);
    __syncthreads();
    stage_parts(stg[0], tpp, rp.in + (long)zc * XY, rp.in + V + (long)zc * ring_plane, tid);
#pragma unroll 1
    for (int k = -4; k < nz; ++k) {
        const int ra1 = ra == 4 ? 0 : ra + 1, ra2 = ra1 == 4 ? 0 : ra1 + 1;
        const int mb1 = mb == 2 ? 0 : mb + 1, mb2 = mb1 == 2 ? 0 : mb1 + 1;
        // (1) density deviation of plane zb+k+2, tile + 2 halo, from the parts
        // staged one iteration ago; stage the parts of plane zb+k+3
        {
            const int cur = (k + 4) & 1;
            cp_async_wait();
            float* out = srho[ra2];
#pragma unroll
            for (int h = 0; h < NRI; ++h) {
                const int e = tid + h * NT;
                if (e < RPAIRS) *reinterpret_cast<float2*>(out + 2 * e) = staged_pair(stg[cur], e, tpp[e]);
            }
            if (k + 1 < nz) {
                const int zn = zc == Z - 1 ? 0 : zc + 1;
                stage_parts(stg[cur ^ 1], tpp, rp.in + (long)zn * XY, rp.in + V + (long)zn * ring_plane, tid);
            }
        }
        __syncthreads();
        // (2) parts streamed by plane zb+k-1; mu pairs of plane zb+k+1, tile + 1 halo
        if (k >= 1) scatter(k - 1);
        if (k >= -2) {
            const float* rm = srho[ra];
            const float* r0 = srho[ra1];
            const float* rpl = srho[ra2];
            float* out = smu[mb2];
#pragma unroll
            for (int j = 0; j < NMU; ++j) {
                const int e = tid + j * NT;
                if (e < MPP) {
                    const int c = 2 * (e % MXP) + OX - 1 + RX * (e / MXP + 1);
                    const F2 rc = F2(r0[c], r0[c + 1]);
                    // sum_i w_i (rho_i - rho) = (1/18) (axis sum) + (1/36) (edge sum) - (2/3) rho
                    // (the Laplacian is 6 times it)
                    F2 sax(0.f), sed(0.f);
#pragma unroll
                    for (int i = 1; i < L::Q; ++i) {
                        const int cz = Vel<L>::cz(i);
                        const float* pl = cz > 0 ? rpl : (cz < 0 ? rm : r0);
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
        // (3) prefetch the pulls of plane zb+k+2; collide the pair of plane
        // zb+k with F = -rho grad mu, store it, and keep its post-collision plane
        if (k >= -2 && k + 2 < nz) {
            const int zp = zb + k + 2;
            const int yv[3] = {wrap_once(y - 1, Y), y, wrap_once(y + 1, Y)};
            const int zv[3] = {XY * wrap_once(zp - 1, Z), XY * zp, XY * wrap_once(zp + 1, Z)};
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const S* p = P.src[i] + X * yv[1 - Vel<L>::cy(i)] + zv[1 - Vel<L>::cz(i)];
                const int cx = Vel<L>::cx(i);
                prefetch_l2(p + (cx == 0 ? x : cx > 0 ? xm : x2));
            }
        }
        if (k >= 0) {
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
            const int yv[3] = {wrap_once(y - 1, Y), y, wrap_once(y + 1, Y)};
            const int zv[3] = {XY * wrap_once(z - 1, Z), XY * z, XY * wrap_once(z + 1, Z)};
            F2 g[L::Q];
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const S* p = P.src[i] + X * yv[1 - Vel<L>::cy(i)] + zv[1 - Vel<L>::cz(i)];
                const int cx = Vel<L>::cx(i);
                if (cx == 0)
                    g[i] = mk2(Acc::plain2(p + x));
                else if (cx > 0)
                    g[i] = F2(Acc::plain1(p + xm), Acc::plain1(p + x));
                else
                    g[i] = F2(Acc::plain1(p + x + 1), Acc::plain1(p + x2));
            }
            if constexpr (SUMS) {
                sum_r += mk2(*reinterpret_cast<const float2*>(srho[ra] + cr));
#pragma unroll
                for (int i = 1; i < L::Q; ++i) {
                    if (Vel<L>::cx(i) > 0) sum_jx += g[i];
                    if (Vel<L>::cx(i) < 0) sum_jx = sum_jx - g[i];
                    if (Vel<L>::cy(i) > 0) sum_jy += g[i];
                    if (Vel<L>::cy(i) < 0) sum_jy = sum_jy - g[i];
                    if (Vel<L>::cz(i) > 0) sum_jz += g[i];
                    if (Vel<L>::cz(i) < 0) sum_jz = sum_jz - g[i];
                }
            }
            const int s = own + XY * z;
            L::collide(g, pre * gx, pre * gy, pre * gz, a.c, (uint32_t)s, a.c.step);
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                g[i] = as_stored<S>(g[i]);
                Acc::store2(P.dst[i] + s, g[i].v);
            }
            put_plane(fpl, g, lx0, ly);
        }
        ra = ra1;
        mb = mb1;
        zc = zc == Z - 1 ? 0 : zc + 1;
    }
    // the last plane's parts, then the top plane (B + S) and the B of the
    // plane above the column (kind 1)
    __syncthreads();
    scatter(nz - 1);
    {
        const int zt = zb + nz - 1;
        *reinterpret_cast<float2*>(rp.out + (long)zt * XY + own) = acc2.v;
        if (tid < NRING) rp.out[V + (long)tile * NRING + tid + (long)zt * ring_plane] = racc2;
        float* e1 = rp.ext + (3L * col + 1) * exs;
        *reinterpret_cast<float2*>(e1 + own) = acc1.v;
        if (tid < NRING) e1[XY + (long)tile * NRING + tid] = racc1;
    }
    if constexpr (SUMS) {
        __shared__ double red[NT / 32][4];
        float v[4] = {sum_r.v.x + sum_r.v.y, sum_jx.v.x + sum_jx.v.y, sum_jy.v.x + sum_jy.v.y,
                      sum_jz.v.x + sum_jz.v.y};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
        if ((tid & 31) == 0)
            for (int q = 0; q < 4; ++q) red[tid >> 5][q] = (double)v[q];
        __syncthreads();
        if (tid < 4) {
            double acc = 0.0;
            for (int w = 0; w < NT / 32; ++w) acc += red[w][tid];
            rows[4 * (blockIdx.x + (long)gridDim.x * (blockIdx.y + (long)gridDim.y * blockIdx.z)) + tid] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Complete the two end planes of every column from the pieces in ext:
//   bottom plane (nz >= 2): ((B from the column below) + S) + A of kind 2
//   top plane (nz >= 2):    (B + S) + A from the column above
//   single-plane column:    ((B from below) + S) + A from above
// One thread per element of a plane's parts (X Y own parts, ntiles 84 ring parts).
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_rho_fixup(T* __restrict__ part, const T* __restrict__ ext, int X, int Y, int Z, int nzc, int ntiles)
{
    const long XY = (long)X * Y;
    const long V = XY * Z;
    const long exs = XY + (long)ntiles * nr::NRING;
    const int ncol = (Z + nzc - 1) / nzc;
    const long n = exs * ncol;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
        const int c = (int)(q / exs);
        const long e = q - (long)c * exs;
        const int zb = c * nzc, nz = min(nzc, Z - zb), ze = zb + nz;
        const int cm = c == 0 ? ncol - 1 : c - 1, cp = c == ncol - 1 ? 0 : c + 1;
        auto at = [&](int z) { return e < XY ? (long)z * XY + e : V + (long)z * ntiles * nr::NRING + (e - XY); };
        const T Bbelow = ext[(3L * cm + 1) * exs + e];
        const T Aabove = ext[(3L * cp + 0) * exs + e];
        if (nz >= 2) {
            const long ib = at(zb), it = at(ze - 1);
            part[ib] = (Bbelow + part[ib]) + ext[(3L * c + 2) * exs + e];
            part[it] = part[it] + Aabove;
        } else {
            const long ib = at(zb);
            part[ib] = (Bbelow + part[ib]) + Aabove;
        }
    }
}

// ---------------------------------------------------------------------------
// The parts of the density of the coming step from stored post-collision
// populations (after flb_init, flb_set_populations, a checkpoint load, ...):
// for every tile and plane t, the same sums as the step forms, each plane in
// one piece.  Block = one tile of one plane; the three source planes t - 1,
// t, t + 1 pass through the post-collision plane in turn.
// ---------------------------------------------------------------------------
template <class S>
__global__ void __launch_bounds__(nr::NT) k_rho_parts(const __grid_constant__ Planes<S> P, float* __restrict__ part,
                                                      int X, int Y, int Z, int ntx)
{
    using namespace nr;
    using Acc = Packed<S>;
    __shared__ __align__(16) float fpl[19 * FP];
    const int tid = threadIdx.x + TXT * threadIdx.y;
    for (int e = tid; e < 19 * FP; e += NT) fpl[e] = 0.f;
    const int lx0 = 2 * threadIdx.x, ly = threadIdx.y;
    const int x = blockIdx.x * TW + lx0, y = blockIdx.y * TH + ly, t = blockIdx.z;
    const long XY = (long)X * Y, V = XY * Z;
    const int ntiles = ntx * (Y / TH);
    int ro[5] = {0, 0, 0, 0, 0};
    if (tid < NRING) ring_sources(tid, ro);
    F2 pc[3];
    float rc[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {  // source plane t - 1 gives B, t gives S, t + 1 gives A
        const int s = q == 0 ? (t == 0 ? Z - 1 : t - 1) : q == 1 ? t : (t == Z - 1 ? 0 : t + 1);
        F2 g[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) g[i] = mk2(Acc::plain2(P.src[i] + x + X * (y + (long)Y * s)));
        __syncthreads();
        put_plane(fpl, g, lx0, ly);
        __syncthreads();
        F2 pS, pB, pA;
        own_pieces(fpl, lx0, ly, pS, pB, pA);
        float rS = 0.f, rB = 0.f, rA = 0.f;
        if (tid < NRING) ring_pieces(fpl, ro, rS, rB, rA);
        pc[q] = q == 0 ? pB : q == 1 ? pS : pA;
        rc[q] = q == 0 ? rB : q == 1 ? rS : rA;
    }
    *reinterpret_cast<float2*>(part + t * XY + x + (long)X * y) = ((pc[0] + pc[1]) + pc[2]).v;
    const int tile = blockIdx.x + ntx * blockIdx.y;
    if (tid < NRING) part[V + ((long)t * ntiles + tile) * NRING + tid] = (rc[0] + rc[1]) + rc[2];
}

}  // namespace flb
