// flb_adjoint.cu -- adjoint (reverse-mode derivative) of one fluctuating LB
// time step of D3Q19, ideal gas or force-based non-ideal fluid, with the
// identical Philox noise replayed.
//
// Forward map of one step, on pre-collision deviations g^n (layout [i][s]):
//   g^{n+1}_i(r + c_i) = C_i(g^n(r), F(r); theta),  F = -rho grad mu,
//   mu = psi'(rho) - kappa lap rho,  rho = rho0 + sum_i g^n_i,
// with C the moment-space collision of Eq. (lbe-mom) (noise included, its
// amplitude depending on the local density).  Given lam^{n+1} = dJ/dg^{n+1}
// the step computes lam^n = dJ/dg^n and adds dJ/dtheta for
// theta = (omega_shear, omega_bulk, omega_ghost, kappa, A, B).
//
// Kernels (per step, all hand-written VJPs):
//   k_adj_collide  pull lam^{n+1}(r + c_i) (adjoint of streaming), replay the
//                  forward collision at r and propagate through it: the local
//                  part of lam^n, the force adjoint Fbar(r) and the relaxation
//                  parameter gradients;
//   k_adj_mu       mubar(y) = -3 sum_i w_i c_i . rho(y - c_i) Fbar(y - c_i)
//                  (adjoint of F = -rho grad mu) and the direct rho term
//                  Fbar . F / rho;
//   k_adj_rho      rhobar = psi''(rho) mubar - kappa lap(mubar) + direct term,
//                  added to every population (rho = sum_i g_i), and the
//                  kappa, A, B gradients.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/flb.h"
#include "flb_internal.h"
#include "flb_prec.cuh"

namespace flb {

Coll<float> coll_fp32(const HostModel& m, uint64_t step);
Coll<double> coll_fp64(const HostModel& m, uint64_t step);

namespace {

using L = D3Q19;

template <class R>
__device__ __forceinline__ R d_sqrt(R x)
{
    return sqrt(x);
}

// Adjoint parameters per launch.
template <class R>
struct AdjArgs {
    Coll<R> c;
    int X, Y, Z;
    long V;
    int nonideal;
    R A, B, kappa, rho0_minus_rhoc, pgrad;
    // d(rel)/d omega = -1/N_a, d(frc)/d omega = -1/(2 N_a), d(ns)/d omega per mode
    R drel[16], dfrc[6], dns[16];
    int cls[16];  // 0 bulk, 1 shear, 2 ghost of non-conserved mode k
};

// Per-site VJP of the collision.  gn: pre-collision deviations at r; F: force
// at r; lb: adjoint of the post-collision populations at r (pulled from step
// n+1).  Out: lg (adjoint of gn, local part), Fb (force adjoint), gp[3]
// (gradients of omega_bulk, omega_shear, omega_ghost).
template <class R>
__device__ __forceinline__ void collide_vjp(const R gn[19], const R F[3], const R lb[19], const AdjArgs<R>& a,
                                            uint32_t site, uint32_t step, R lg[19], R Fb[3], R gp[3])
{
    const Coll<R>& P = a.c;
    R m[19];
    L::moments(gn, m);
    const R rho = P.rho0 + m[0];
    const R ir = R(1) / rho;
    const R ux = (m[1] + R(0.5) * F[0]) * ir, uy = (m[2] + R(0.5) * F[1]) * ir, uz = (m[3] + R(0.5) * F[2]) * ir;
    const R Fx = F[0], Fy = F[1], Fz = F[2];
    const R uxx = ux * ux, uyy = uy * uy, uzz = uz * uz, uu = uxx + uyy + uzz;
    const R uF = ux * Fx + uy * Fy + uz * Fz;
    R z[16];
    R sr = R(0), dsr = R(0);  // noise amplitude factor and its rho derivative
    if (P.noise) {
        noise_normals<4>(P.key, site, step, P.replica, z);
        if (P.noise_local) {
            sr = d_sqrt(rho);
            dsr = R(0.5) / sr;
        } else {
            sr = P.sqrt_rho0;
        }
    } else {
        for (int k = 0; k < 16; ++k) z[k] = R(0);
    }
    // adjoint of the increments: Db_a = sum_i w_i T_ai lb_i
    R wl[19], Db[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) wl[i] = R(Vel<L>::w(i)) * lb[i];
    L::moments(wl, Db);

    // forward pieces needed for the parameter gradients
    const R neq[6] = {m[4] - rho * uu, m[5] - rho * (R(3) * uxx - uu), m[6] - rho * (uyy - uzz),
                      m[7] - rho * ux * uy, m[8] - rho * uy * uz, m[9] - rho * uz * ux};
    const R mF[6] = {R(2) * uF, R(2) * (R(3) * ux * Fx - uF), R(2) * (uy * Fy - uz * Fz),
                     ux * Fy + uy * Fx, uy * Fz + uz * Fy, uz * Fx + ux * Fz};

    R mb[19];  // adjoint of the moments
    R rb = R(0), ubx = R(0), uby = R(0), ubz = R(0);
    R fbx = R(3) * Db[1], fby = R(3) * Db[2], fbz = R(3) * Db[3];
    gp[0] = gp[1] = gp[2] = R(0);
#pragma unroll
    for (int k = 0; k < 15; ++k) {
        const int aidx = 4 + k;
        const R d = Db[aidx];
        mb[aidx] = P.rel[k] * d;
        // parameter gradient of this mode
        R g = a.drel[k] * (k < 6 ? neq[k] : m[aidx]) + a.dns[k] * sr * z[k];
        if (k < 6) g += a.dfrc[k] * mF[k];
        gp[a.cls[k]] += d * g;
        // noise amplitude through rho
        rb += d * P.ns[k] * z[k] * dsr;
    }
    const R* rl = P.rel;
    const R* fr = P.frc;
    const R d4 = Db[4], d5 = Db[5], d6 = Db[6], d7 = Db[7], d8 = Db[8], d9 = Db[9];
    // d/drho at fixed u of the equilibrium parts
    rb += -rl[0] * uu * d4 - rl[1] * (R(3) * uxx - uu) * d5 - rl[2] * (uyy - uzz) * d6 - rl[3] * ux * uy * d7 -
          rl[4] * uy * uz * d8 - rl[5] * uz * ux * d9;
    // d/du
    ubx += d4 * (R(-2) * rl[0] * rho * ux + R(2) * fr[0] * Fx) + d5 * (R(-4) * rl[1] * rho * ux + R(4) * fr[1] * Fx) +
           d7 * (-rl[3] * rho * uy + fr[3] * Fy) + d9 * (-rl[5] * rho * uz + fr[5] * Fz);
    uby += d4 * (R(-2) * rl[0] * rho * uy + R(2) * fr[0] * Fy) + d5 * (R(2) * rl[1] * rho * uy - R(2) * fr[1] * Fy) +
           d6 * (R(-2) * rl[2] * rho * uy + R(2) * fr[2] * Fy) + d7 * (-rl[3] * rho * ux + fr[3] * Fx) +
           d8 * (-rl[4] * rho * uz + fr[4] * Fz);
    ubz += d4 * (R(-2) * rl[0] * rho * uz + R(2) * fr[0] * Fz) + d5 * (R(2) * rl[1] * rho * uz - R(2) * fr[1] * Fz) +
           d6 * (R(2) * rl[2] * rho * uz - R(2) * fr[2] * Fz) + d8 * (-rl[4] * rho * uy + fr[4] * Fy) +
           d9 * (-rl[5] * rho * ux + fr[5] * Fx);
    // d/dF at fixed u
    fbx += d4 * R(2) * fr[0] * ux + d5 * R(4) * fr[1] * ux + d7 * fr[3] * uy + d9 * fr[5] * uz;
    fby += d4 * R(2) * fr[0] * uy - d5 * R(2) * fr[1] * uy + d6 * R(2) * fr[2] * uy + d7 * fr[3] * ux + d8 * fr[4] * uz;
    fbz += d4 * R(2) * fr[0] * uz - d5 * R(2) * fr[1] * uz - d6 * R(2) * fr[2] * uz + d8 * fr[4] * uy + d9 * fr[5] * ux;
    // u = (j + F/2) / rho
    mb[1] = ubx * ir;
    mb[2] = uby * ir;
    mb[3] = ubz * ir;
    fbx += R(0.5) * ubx * ir;
    fby += R(0.5) * uby * ir;
    fbz += R(0.5) * ubz * ir;
    rb -= (ubx * ux + uby * uy + ubz * uz) * ir;
    mb[0] = rb;
    // lg = lb + T^T mb  (T^T mb = from_moments(mb) / w)
    R t[19];
    L::from_moments(mb, t);
#pragma unroll
    for (int i = 0; i < 19; ++i) lg[i] = lb[i] + t[i] * R(1.0 / Vel<L>::w(i));
    Fb[0] = fbx;
    Fb[1] = fby;
    Fb[2] = fbz;
}

__device__ __forceinline__ long blin() { return blockIdx.x + (long)gridDim.x * (blockIdx.y + (long)gridDim.y * blockIdx.z); }

// Block sums of NV per-thread values: warp sums in the compute type (32
// terms; FP64 arithmetic per thread would run on GB300's slow FP64 pipe),
// then FP64 across the warps of the block and, in sum_columns, across blocks.
template <int NV, class R>
__device__ __forceinline__ void block_rows(R v[NV], double* __restrict__ row)
{
    __shared__ double red[32][NV];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if ((tid & 31) == 0)
        for (int k = 0; k < NV; ++k) red[tid >> 5][k] = (double)v[k];
    __syncthreads();
    for (int k = tid; k < NV; k += nthr) {
        double acc = 0.0;
        for (int w = 0; w < (nthr + 31) / 32; ++w) acc += red[w][k];
        row[k] = acc;
    }
}

// densities and forces of the state g^n (pre-collision deviations)
template <class R>
__global__ void k_adj_rho(const R* __restrict__ gn, R* __restrict__ drho, long V)
{
    for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < V; s += (long)gridDim.x * blockDim.x) {
        R g[19], m[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) g[i] = gn[(long)i * V + s];
        L::moments(g, m);
        drho[s] = m[0];
    }
}

// rb_next (or NULL): the density part of lam_next kept apart by the previous
// adjoint step of a segment; lam_next + rb_next is the full adjoint state.
template <class R>
__global__ void k_adj_collide(const AdjArgs<R> a, uint32_t step, const R* __restrict__ gn, const R* __restrict__ F,
                              const R* __restrict__ lam_next, const R* __restrict__ rb_next, R* __restrict__ lam,
                              R* __restrict__ Fbar, double* __restrict__ rows)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    R gp[3] = {R(0), R(0), R(0)};
    if (x < a.X && y < a.Y && z < a.Z) {
        const long V = a.V;
        const int s = x + a.X * (y + a.Y * z);
        const Nbhd nb(x, y, z, a.X, a.Y, a.Z);
        R g[19], lb[19], lg[19], Fs[3] = {R(0), R(0), R(0)}, Fb[3];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            g[i] = gn[(long)i * V + s];
            // streaming moved the post-collision population i from r to r + c_i
            const int q = nb.src(-Vel<L>::cx(i), -Vel<L>::cy(i), -Vel<L>::cz(i));
            lb[i] = rb_next ? lam_next[(long)i * V + q] + rb_next[q] : lam_next[(long)i * V + q];
        }
        if (a.nonideal)
            for (int d = 0; d < 3; ++d) Fs[d] = F[d * V + s];
        collide_vjp(g, Fs, lb, a, (uint32_t)s, step, lg, Fb, gp);
#pragma unroll
        for (int i = 0; i < 19; ++i) lam[(long)i * V + s] = lg[i];
        if (a.nonideal)
            for (int d = 0; d < 3; ++d) Fbar[d * V + s] = Fb[d];
    }
    block_rows<3>(gp, rows + blin() * 6);
}

// F(r) = -rho(r) grad mu(r) + pgrad sum_i w_i c_i rho(r + c_i).  Adjoint:
// mubar(y) = -3 sum_i w_i c_i . rho(y - c_i) Fbar(y - c_i);
// rb1(y) = Fbar(y) . (-grad mu(y)) + pgrad sum_i w_i c_i . Fbar(y - c_i),
// with -grad mu(y) = (F(y) - pgrad sum_i w_i c_i rho(y + c_i)) / rho(y).
template <class R>
__global__ void k_adj_mu(const AdjArgs<R> a, const R* __restrict__ drho, const R* __restrict__ F,
                         const R* __restrict__ Fbar, R* __restrict__ mubar, R* __restrict__ rb1)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x >= a.X || y >= a.Y || z >= a.Z) return;
    const long V = a.V;
    const int s = x + a.X * (y + a.Y * z);
    const Nbhd nb(x, y, z, a.X, a.Y, a.Z);
    R acc = R(0), accp = R(0), pr[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int q = nb.src(Vel<L>::cx(i), Vel<L>::cy(i), Vel<L>::cz(i));  // y - c_i
        const R rq = a.c.rho0 + drho[q];
        const R cf = Vel<L>::cx(i) * Fbar[q] + Vel<L>::cy(i) * Fbar[V + q] + Vel<L>::cz(i) * Fbar[2 * V + q];
        acc += R(Vel<L>::w(i)) * rq * cf;
        accp += R(Vel<L>::w(i)) * cf;
        const R wr = R(Vel<L>::w(i)) * drho[nb.src(-Vel<L>::cx(i), -Vel<L>::cy(i), -Vel<L>::cz(i))];  // y + c_i
        pr[0] += R(Vel<L>::cx(i)) * wr;
        pr[1] += R(Vel<L>::cy(i)) * wr;
        pr[2] += R(Vel<L>::cz(i)) * wr;
    }
    mubar[s] = R(-3) * acc;
    const R rho = a.c.rho0 + drho[s];
    R fg = R(0);
    for (int d = 0; d < 3; ++d) fg += Fbar[d * V + s] * (F[d * V + s] - a.pgrad * pr[d]);
    rb1[s] = fg / rho + a.pgrad * accp;
}

// rhobar = rb1 + psi''(rho) mubar - kappa lap(mubar), added to every population
// (or, with rb_out, stored for the next adjoint step of a segment to add);
// kappa, A, B gradients
template <class R>
__global__ void k_adj_rho(const AdjArgs<R> a, const R* __restrict__ drho, const R* __restrict__ mubar,
                          const R* __restrict__ rb1, R* __restrict__ lam, R* __restrict__ rb_out,
                          double* __restrict__ rows)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    R gp[3] = {R(0), R(0), R(0)};
    if (x < a.X && y < a.Y && z < a.Z) {
        const long V = a.V;
        const int s = x + a.X * (y + a.Y * z);
        const Nbhd nb(x, y, z, a.X, a.Y, a.Z);
        const R mb = mubar[s], r0 = drho[s];
        R lapm = R(0), lapr = R(0);
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const int q = nb.src(-Vel<L>::cx(i), -Vel<L>::cy(i), -Vel<L>::cz(i));  // y + c_i
            lapm += R(Vel<L>::w(i)) * (mubar[q] - mb);
            lapr += R(Vel<L>::w(i)) * (drho[q] - r0);
        }
        lapm *= R(6);
        lapr *= R(6);
        const R d = r0 + a.rho0_minus_rhoc;
        const R psi2 = a.A + R(3) * a.B * d * d;
        const R rb = rb1[s] + psi2 * mb - a.kappa * lapm;
        if (rb_out)
            rb_out[s] = rb;
        else
#pragma unroll
            for (int i = 0; i < 19; ++i) lam[(long)i * V + s] += rb;
        gp[0] = -mb * lapr;   // kappa
        gp[1] = mb * d;       // A
        gp[2] = mb * d * d * d;  // B
    }
    block_rows<3>(gp, rows + blin() * 6 + 3);
}

// lam += rb on every population: the deferred density part of the last step
template <class R>
__global__ void k_add_rb(R* __restrict__ lam, const R* __restrict__ rb, long V)
{
    for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < V; s += (long)gridDim.x * blockDim.x) {
        const R r = rb[s];
#pragma unroll
        for (int i = 0; i < 19; ++i) lam[(long)i * V + s] += r;
    }
}

// Column c of the per-block rows summed (in the order of k_sum_columns) and
// added to its parameter: columns (bulk, shear, ghost, kappa, A, B) go to
// grad (omega_shear, omega_bulk, omega_ghost, kappa, A, B).  One block per
// column; the free-energy columns only for the non-ideal fluid.
__global__ void k_add_grads(const double* __restrict__ rows, int nrows, double* __restrict__ grad, int nonideal)
{
    __shared__ double sh[256];
    const int c = blockIdx.x;
    if (c >= 3 && !nonideal) return;
    double acc = 0.0;
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) acc += rows[(long)r * 6 + c];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) grad[c == 0 ? 1 : c == 1 ? 0 : c] += sh[0];
}

template <class R>
AdjArgs<R> make_adj(const HostModel& m, const Coll<R>& c)
{
    AdjArgs<R> a{};
    a.c = c;
    a.X = m.X;
    a.Y = m.Y;
    a.Z = m.Z;
    a.V = m.V;
    a.nonideal = m.nonideal;
    a.A = R(m.A);
    a.B = R(m.B);
    a.kappa = R(m.kappa);
    a.rho0_minus_rhoc = R(m.rho0 - m.rho_c);
    a.pgrad = R(m.nonideal && m.total ? 1 : 0);
    for (int k = 0; k < 15; ++k) {
        const int aidx = 4 + k;
        const double om = k == 0 ? m.om_b : k < 6 ? m.om_s : m.om_g;
        const double Na = L::N(aidx);
        a.cls[k] = k == 0 ? 0 : k < 6 ? 1 : 2;
        a.drel[k] = R(-1.0 / Na);
        if (k < 6) a.dfrc[k] = R(-0.5 / Na);
        const double ns = std::sqrt(m.kT * (2.0 - om) * om * Na * 3.0) / Na;
        a.dns[k] = R(ns * (1.0 - om) / (om * (2.0 - om)));
    }
    return a;
}

template <class R>
cudaError_t adjoint_step_t(const HostModel& m, const Coll<R>& c, uint64_t step, const R* gn, const R* lam_next,
                           const R* rb_next, R* lam, R* rb_out, R* work, double* rows, double* grad,
                           cudaStream_t st)
{
    const long V = m.V;
    R* drho = work;
    R* mu = work + V;
    R* F = work + 2 * V;
    R* Fbar = work + 5 * V;
    R* mubar = work + 8 * V;
    R* rb1 = work + 9 * V;
    const AdjArgs<R> a = make_adj<R>(m, c);
    const dim3 b(32, 4, 2);
    const dim3 g((m.X + 31) / 32, (m.Y + 3) / 4, (m.Z + 1) / 2);
    const int nrows = (int)(g.x * g.y * g.z);
    cudaError_t e = cudaSuccess;
    // every block writes columns 0-2 (collision) and, for the non-ideal fluid,
    // 3-5 (free-energy parameters); the ideal gas leaves 3-5 at zero
    if (!m.nonideal && (e = cudaMemsetAsync(rows, 0, (size_t)nrows * 6 * sizeof(double), st)) != cudaSuccess)
        return e;
    if (m.nonideal) {
        k_adj_rho<R><<<(unsigned)std::min<long>((V + 255) / 256, 152 * 16), 256, 0, st>>>(gn, drho, V);
        StepArgs<R> sa{};
        sa.c = c;
        sa.X = m.X;
        sa.Y = m.Y;
        sa.Z = m.Z;
        sa.V = V;
        sa.A = a.A;
        sa.B = a.B;
        sa.kappa = a.kappa;
        sa.rho0_minus_rhoc = a.rho0_minus_rhoc;
        sa.pgrad = a.pgrad;
        k_mu<L, R><<<g, b, 0, st>>>(sa, drho, mu);
        k_force<L, R><<<g, b, 0, st>>>(sa, drho, mu, F);
    }
    k_adj_collide<R><<<g, b, 0, st>>>(a, (uint32_t)step, gn, F, lam_next, rb_next, lam, Fbar, rows);
    if (m.nonideal) {
        k_adj_mu<R><<<g, b, 0, st>>>(a, drho, F, Fbar, mubar, rb1);
        k_adj_rho<R><<<g, b, 0, st>>>(a, drho, mubar, rb1, lam, rb_out, rows);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_add_grads<<<6, 256, 0, st>>>(rows, nrows, grad, m.nonideal);
    return cudaGetLastError();
}

}  // namespace

cudaError_t adjoint_step(const HostModel& m, int prec, uint64_t step, const void* gn, const void* lam_next,
                         const void* rb_next, void* lam, void* rb_out, void* work, double* rows, double* grad,
                         cudaStream_t st)
{
    if (prec == FLB_FP64)
        return adjoint_step_t<double>(m, coll_fp64(m, step), step, (const double*)gn, (const double*)lam_next,
                                      (const double*)rb_next, (double*)lam, (double*)rb_out, (double*)work, rows,
                                      grad, st);
    return adjoint_step_t<float>(m, coll_fp32(m, step), step, (const float*)gn, (const float*)lam_next,
                                 (const float*)rb_next, (float*)lam, (float*)rb_out, (float*)work, rows, grad,
                                 st);
}

cudaError_t adjoint_add_rb(const HostModel& m, int prec, void* lam, const void* rb, cudaStream_t st)
{
    const unsigned nb = (unsigned)std::min<long>((m.V + 255) / 256, 152 * 16);
    if (prec == FLB_FP64)
        k_add_rb<double><<<nb, 256, 0, st>>>((double*)lam, (const double*)rb, m.V);
    else
        k_add_rb<float><<<nb, 256, 0, st>>>((float*)lam, (const float*)rb, m.V);
    return cudaGetLastError();
}

int adjoint_rows(const HostModel& m)
{
    return ((m.X + 31) / 32) * ((m.Y + 3) / 4) * ((m.Z + 1) / 2);
}

}  // namespace flb
