// flb_noalloc.cu -- structure factor that allocates nothing.
//
// Some callers cannot allocate device memory while they run: hosts whose
// allocator forbids cudaMalloc after start-up (a serving process that sizes
// its device memory once), real-time loops whose memory budget is fixed up
// front, or code running where an allocation would synchronise the device.
// This entry point gives them the structure factor of flb_structure_factor
// from device buffers they already own; its FFT work array is a file-scope
// static device array instead of memory obtained from cudaMalloc.
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

// Per device, looked up once with that device current: the device address of
// g_sf_work (in host code the symbol is a host-side stand-in, not an address)
// and the number of SMs, which sizes the grid.  The entries live until the
// process exits; a cudaDeviceReset by the caller invalidates them.
constexpr int kMaxDevices = 128;
struct DeviceSlot {
    double2* work;
    int sms;
};
DeviceSlot g_slot[kMaxDevices] = {};
std::mutex g_slot_mutex;

cudaError_t device_slot(int dev, DeviceSlot* out)
{
    std::lock_guard<std::mutex> lock(g_slot_mutex);
    DeviceSlot& d = g_slot[dev];
    if (!d.work) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_sf_work);
        if (e != cudaSuccess) return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        d.sms = sms > 0 ? sms : 1;
        d.work = static_cast<double2*>(p);
    }
    *out = d;
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
    // edges first: each is then at most 4096, so their product fits in a long
    for (int d = 0; d < 3; ++d)
        if (!flb::fft_length_in_place(dims[d]))
            return flb::set_error(FLB_EINVAL, "edge length " + std::to_string(dims[d]) +
                                                  " is not a product of 2, 3 and 5 (up to 4096)");
    const long V = (long)dims[0] * dims[1] * dims[2];
    if (V > FLB_NOALLOC_MAX_SITES)
        return flb::set_error(FLB_EINVAL, "lattice has " + std::to_string(V) + " sites; the allocation-free "
                                          "structure factor handles at most FLB_NOALLOC_MAX_SITES = " +
                                              std::to_string(FLB_NOALLOC_MAX_SITES));
    if (mode < 0 || mode >= lattice) return flb::set_error(FLB_EINVAL, "mode out of range");

    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return flb::set_error(FLB_ECUDA, std::string("no usable current device: ") + cudaGetErrorString(e));
    DeviceSlot slot;
    e = device_slot(dev, &slot);
    if (e != cudaSuccess)
        return flb::set_error(FLB_ECUDA, std::string("device set-up of the work array: ") + cudaGetErrorString(e));
    double2* work = slot.work;

    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    long nb = (V + 255) / 256;
    if (nb > 16L * slot.sms) nb = 16L * slot.sms;
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
