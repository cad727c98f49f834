// flb_capillary.cu -- interface heights and height spectrum of a liquid stripe.
//
// Capillary fluctuations (Sec. VI): the height h(x) of an interface is the
// shift of the intrinsic mean-field profile that matches the instantaneous
// density of column x (Eq. (height-def)), with the profile of Eq. (denprof)
//   rho_MF(s) = (rho_L + rho_V)/2 +- (rho_L - rho_V)/2 tanh(2 s / w).
// The fit is a least-squares match over a window of rows, solved for h by
// Gauss-Newton; the spectrum |h(k)|^2 / X is then compared with
// kT / (sigma (2 - 2 cos k)) (Eq. (capill-static) on the lattice).
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/flb.h"
#include "flb_internal.h"

namespace flb {
namespace {

// One thread per (column, interface): interface 0 is the lower one (vapour
// below, liquid above, profile rising with y), interface 1 the upper one.
template <class R>
__global__ void k_heights(const R* __restrict__ drho, double rho0, int X, int Y, const flb_interface_fit f,
                          double* __restrict__ h)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * X) return;
    const int x = t % X, which = t / X;
    const double sgn = which == 0 ? 1.0 : -1.0;
    const double mid = 0.5 * (f.rho_l + f.rho_v), amp = 0.5 * (f.rho_l - f.rho_v);
    const double k2 = 2.0 / f.width;
    const int c = (int)llrint(f.guess[which]);
    double hh = f.guess[which];
    for (int it = 0; it < f.iterations; ++it) {
        double jj = 0.0, jr = 0.0;
        for (int yy = c - f.window; yy <= c + f.window; ++yy) {
            int y = yy % Y;
            if (y < 0) y += Y;
            const double rho = rho0 + (double)drho[x + (long)X * y];
            const double th = tanh(k2 * (yy - hh));
            const double r = rho - (mid + sgn * amp * th);
            const double j = -sgn * amp * k2 * (1.0 - th * th);  // d rho_MF / d h
            jj += j * j;
            jr += j * r;
        }
        hh += jr / jj;
    }
    h[t] = hh;
}

// Line i of 2: data = h - mean(h) as complex numbers (one block per line).
__global__ void k_center_lines(const double* __restrict__ h, int X, double2* __restrict__ data)
{
    __shared__ double part[256];
    const double* line = h + (long)blockIdx.x * X;
    double s = 0.0;
    for (int x = threadIdx.x; x < X; x += blockDim.x) s += line[x];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    const double mean = part[0] / X;
    for (int x = threadIdx.x; x < X; x += blockDim.x)
        data[(long)blockIdx.x * X + x] = make_double2(line[x] - mean, 0.0);
}

// p(k) = (|H_0(k)|^2 + |H_1(k)|^2) / (2 X); accumulate: acc += p, else out = p.
__global__ void k_height_power(const double2* __restrict__ d, int X, double* __restrict__ acc,
                               double* __restrict__ out)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < X; k += gridDim.x * blockDim.x) {
        const double2 a = d[k], b = d[X + k];
        const double p = (a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y) / (2.0 * X);
        if (acc)
            acc[k] += p;
        else
            out[k] = p;
    }
}

}  // namespace

cudaError_t interface_heights(const void* drho, int real_size, double rho0, int X, int Y,
                              const flb_interface_fit& f, double* h, cudaStream_t s)
{
    const int n = 2 * X, b = 128;
    if (real_size == 8)
        k_heights<double><<<(n + b - 1) / b, b, 0, s>>>((const double*)drho, rho0, X, Y, f, h);
    else
        k_heights<float><<<(n + b - 1) / b, b, 0, s>>>((const float*)drho, rho0, X, Y, f, h);
    return cudaGetLastError();
}

cudaError_t height_power(const double* h, int X, double2* work, double2* scratch, double* acc, double* out,
                         cudaStream_t s)
{
    k_center_lines<<<2, 256, 0, s>>>(h, X, work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = fft_rows(work, X, 2, scratch, s)) != cudaSuccess) return e;
    k_height_power<<<(X + 255) / 256, 256, 0, s>>>(work, X, acc, out);
    return cudaGetLastError();
}

}  // namespace flb
