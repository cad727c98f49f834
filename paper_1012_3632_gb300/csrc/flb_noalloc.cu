// flb_noalloc.cu -- structure factor that allocates nothing.
//
// Some callers cannot allocate device memory while they run: code that is
// captured into a CUDA graph, hosts whose allocator forbids cudaMalloc after
// start-up, or real-time loops whose memory budget is fixed up front.  This
// entry point gives them the structure factor of flb_structure_factor from
// device buffers they already own; its FFT work array is a file-scope static
// device array instead of memory obtained from cudaMalloc.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/flb.h"
#include "flb_device.cuh"
#include "flb_internal.h"

namespace {

// FFT work array shared by every call (16 MiB of complex doubles).  Every GPU
// that loads the library keeps it until the process exits.
__device__ __align__(256) double2 g_sf_work[FLB_NOALLOC_MAX_SITES];

// Device address of g_sf_work per device, looked up once with that device
// current (in host code the symbol is a host-side stand-in, not an address).
constexpr int kMaxDevices = 128;
double2* g_work_addr[kMaxDevices] = {nullptr};
std::mutex g_work_mutex;

cudaError_t work_address(int dev, double2** out)
{
    std::lock_guard<std::mutex> lock(g_work_mutex);
    if (!g_work_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_sf_work);
        if (e != cudaSuccess) return e;
        g_work_addr[dev] = static_cast<double2*>(p);
    }
    *out = g_work_addr[dev];
    return cudaSuccess;
}

// m_mode(r) = sum_i T_ai f_i(r) of pre-collision populations f[i*V + s].
template <class L>
__global__ void k_mode_of_populations(const double* __restrict__ f, int mode, double2* __restrict__ out, long V)
{
    for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < V; s += (long)gridDim.x * blockDim.x) {
        double g[L::Q], m[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) g[i] = f[(long)i * V + s];
        L::moments(g, m);
        double v = m[0];
#pragma unroll
        for (int q = 1; q < L::Q; ++q)
            if (q == mode) v = m[q];
        out[s] = make_double2(v, 0.0);
    }
}

}  // namespace

extern "C" int flb_structure_factor_noalloc(int lattice, const int dims[3], const double* f, int mode, double* S,
                                            void* stream)
{
    FLB_TRACE();
    if (lattice != FLB_D2Q9 && lattice != FLB_D3Q19)
        return flb::set_error(FLB_EINVAL, "lattice must be FLB_D2Q9 or FLB_D3Q19");
    if (!dims || !f || !S) return flb::set_error(FLB_EINVAL, "dims, f and S must not be NULL");
    for (int d = 0; d < 3; ++d)
        if (dims[d] < 1) return flb::set_error(FLB_EINVAL, "every dimension must be >= 1");
    if (lattice == FLB_D2Q9 && dims[2] != 1) return flb::set_error(FLB_EINVAL, "D2Q9 needs dims[2] == 1");
    const long V = (long)dims[0] * dims[1] * dims[2];
    if (V > FLB_NOALLOC_MAX_SITES)
        return flb::set_error(FLB_EINVAL, "lattice has " + std::to_string(V) + " sites; the allocation-free "
                                          "structure factor handles at most FLB_NOALLOC_MAX_SITES = " +
                                              std::to_string(FLB_NOALLOC_MAX_SITES));
    for (int d = 0; d < 3; ++d)
        if (!flb::fft_length_in_place(dims[d]))
            return flb::set_error(FLB_EINVAL, "edge length " + std::to_string(dims[d]) +
                                                  " is not a product of 2, 3 and 5 (up to 4096)");
    if (mode < 0 || mode >= lattice) return flb::set_error(FLB_EINVAL, "mode out of range");

    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return flb::set_error(FLB_ECUDA, std::string("no usable current device: ") + cudaGetErrorString(e));
    double2* work = nullptr;
    e = work_address(dev, &work);
    if (e != cudaSuccess)
        return flb::set_error(FLB_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));

    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    long nb = (V + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    if (lattice == FLB_D3Q19)
        k_mode_of_populations<flb::D3Q19><<<(unsigned)nb, 256, 0, st>>>(f, mode, work, V);
    else
        k_mode_of_populations<flb::D2Q9><<<(unsigned)nb, 256, 0, st>>>(f, mode, work, V);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = flb::fft3d(work, dims[0], dims[1], dims[2], nullptr, st);
    if (e == cudaSuccess) e = flb::power_spectrum(work, V, nullptr, S, st);
    if (e != cudaSuccess)
        return flb::set_error(FLB_ECUDA, std::string("flb_structure_factor_noalloc: ") + cudaGetErrorString(e));
    return FLB_OK;
}
