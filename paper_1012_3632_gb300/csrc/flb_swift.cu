// flb_swift.cu -- the k-dependent noise of the modified-equilibrium model.
//
// Sec. IV.C: with the non-ideal pressure in the equilibrium (Eq. (meq-yeo)),
// the FDT of Eq. (dbe-fdt) gives a noise whose covariance depends on the
// wavevector and couples the bulk mode e with the ghost mode eps
// (Eq. (noise-yeo)).  On the lattice (Sec. V: xi^LB = (1 - omega/2) xi with
// lambda = 2 omega / (2 - omega)) the per-site, per-step covariance of
// (xi_e, xi_eps) at wavevector k is
//   C_ee  = s_e^2   P N_e   (2 - 3 c2(k)) lambda_e,
//   C_pp  = s_eps^2 P N_eps (5/4 - 3/4 c2(k)) lambda_eps,
//   C_ep  = s_e s_eps P 6 (c2(k) - cs^2)(lambda_e + lambda_eps),
// P = 2 rho0 kT / cs^2, s = 1 - omega/2, c2(k) = dp0/drho(rho0) + kappa rho0 K2(k),
// K2(k) = (2/cs^2) sum_i w_i (1 - cos k.c_i) (the symbol of -lap).  The corner
// is printed with 12; the FDT with Eqs. (FDBE-yeo), (meq-yeo), (f-correl-yeo)
// gives 6, and with 6 the covariance of Eq. (f-correl-yeo) is the exact
// stationary state of the linear lattice update.
//
// The noise is coloured in Fourier space: white normals z_e(r), z_eps(r) (the
// collision's own Philox draw for the modes e and eps), Z = FFT(z_e + i z_eps),
// per k the pair (E, P) = ((Z(k) + Z*(-k))/2, (Z(k) - Z*(-k))/(2i)) is
// multiplied by the lower Cholesky factor of C(k), and an FFT of the conjugate
// gives V times the conjugate of the inverse transform.  FP64 storage
// colours the noise with FP64 transforms, FP32 and BF16 storage with FP32
// transforms (a random field that needs no more precision).
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/flb.h"
#include "flb_device.cuh"
#include "flb_internal.h"

namespace flb {
namespace {

// Z(r) = z_e(r) + i z_eps(r): normals 0 and 5 of the D2Q9 collision draw
// (calls 0 and 1 of tag 0), stored as T: Box-Muller in FP64 for double2 and in
// FP32 for float2, as the collision kernels of those precisions draw them.
template <class T>
__global__ void k_swift_white(PhiloxKeys key, uint32_t step, uint32_t replica, long V, T* __restrict__ Z)
{
    using E = decltype(T::x);
    for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < V; s += (long)gridDim.x * blockDim.x) {
        E a[4], b[4];
        normals4<E>(key, (uint32_t)s, step, 0u, replica, a);
        normals4<E>(key, (uint32_t)s, step, 1u, replica, b);
        Z[s] = T{a[0], b[1]};
    }
}

// out(k) = conj(Ze'(k) + i Zp'(k)) with (Ze', Zp') = chol(k) (E, P).
template <class T>
__global__ void k_swift_colour(const T* __restrict__ Z, const double* __restrict__ chol, int X, int Y,
                               T* __restrict__ out)
{
    using E = decltype(T::x);
    const long V = (long)X * Y;
    for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < V; s += (long)gridDim.x * blockDim.x) {
        const int nx = (int)(s % X), ny = (int)(s / X);
        const long sm = (long)((X - nx) % X) + (long)X * ((Y - ny) % Y);  // -k
        const T zk = Z[s], zm = Z[sm];
        // E = (Z(k) + conj Z(-k)) / 2, P = (Z(k) - conj Z(-k)) / (2i)
        const E er = E(0.5) * (zk.x + zm.x), ei = E(0.5) * (zk.y - zm.y);
        const E pr = E(0.5) * (zk.y + zm.y), pi = E(-0.5) * (zk.x - zm.x);
        const E c11 = E(chol[3 * s]), c21 = E(chol[3 * s + 1]), c22 = E(chol[3 * s + 2]);
        const E Er = c11 * er, Ei = c11 * ei;
        const E Pr = c21 * er + c22 * pr, Pi = c21 * ei + c22 * pi;
        // E' + i P' = (Er - Pi) + i (Ei + Pr); conjugate
        out[s] = T{Er - Pi, -(Ei + Pr)};
    }
}

template <class T>
cudaError_t swift_noise_t(const HostModel& m, uint64_t step, const double* chol, T* work, T* out, cudaStream_t s)
{
    const long V = m.V;
    const unsigned nb = (unsigned)std::min<long>((V + 255) / 256, 152 * 16);
    k_swift_white<T><<<nb, 256, 0, s>>>(philox_keys(m.seed), (uint32_t)step, m.replica, V, work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = fft3d(work, m.X, m.Y, 1, out, s)) != cudaSuccess) return e;
    k_swift_colour<T><<<nb, 256, 0, s>>>(work, chol, m.X, m.Y, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return fft3d(out, m.X, m.Y, 1, work, s);
}

}  // namespace

bool swift_table(const HostModel& m, double* chol, std::string& err)
{
    const double cs2 = 1.0 / 3.0, pi = 3.14159265358979323846;
    const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const double d = m.rho0 - m.rho_c;
    const double c2_0 = m.rho0 * (m.A + 3.0 * m.B * d * d) + (m.total ? 0.0 : cs2);
    const double oe = m.om_b, op = m.om_g;
    const double le = 2.0 * oe / (2.0 - oe), lp = 2.0 * op / (2.0 - op);
    const double se = 1.0 - 0.5 * oe, sp = 1.0 - 0.5 * op;
    const double P = 2.0 * m.rho0 * m.kT / cs2;
    const double Ne = 4.0, Np = 16.0;
    for (int ny = 0; ny < m.Y; ++ny)
        for (int nx = 0; nx < m.X; ++nx) {
            const double kx = 2.0 * pi * nx / m.X, ky = 2.0 * pi * ny / m.Y;
            double K2 = 0.0;
            for (int i = 0; i < 9; ++i) K2 += w[i] * (1.0 - std::cos(kx * cx[i] + ky * cy[i]));
            K2 *= 2.0 / cs2;
            const double c2 = c2_0 + m.kappa * m.rho0 * K2;
            const double a = se * se * P * Ne * (2.0 - 3.0 * c2) * le;
            const double c = sp * sp * P * Np * (1.25 - 0.75 * c2) * lp;
            const double b = se * sp * P * 6.0 * (c2 - cs2) * (le + lp);
            const long s = nx + (long)m.X * ny;
            if (!(a > 0.0) || !(c - b * b / a >= 0.0)) {
                err = "modified-equilibrium noise covariance is not positive definite at k = (" + std::to_string(kx) +
                      ", " + std::to_string(ky) + "), c_s^2(k) = " + std::to_string(c2);
                return false;
            }
            const double c11 = std::sqrt(a), c21 = b / c11;
            chol[3 * s] = c11;
            chol[3 * s + 1] = c21;
            chol[3 * s + 2] = std::sqrt(std::max(c - c21 * c21, 0.0));
        }
    return true;
}

cudaError_t swift_noise(const HostModel& m, uint64_t step, const double* chol, void* work, void* out, bool fp32,
                        cudaStream_t s)
{
    if (fp32) return swift_noise_t(m, step, chol, (float2*)work, (float2*)out, s);
    return swift_noise_t(m, step, chol, (double2*)work, (double2*)out, s);
}

}  // namespace flb
