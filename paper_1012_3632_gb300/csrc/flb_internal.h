// flb_internal.h -- host-side interface between the C ABI (flb_api.cu) and the
// precision-specific kernel instantiations (flb_fp64.cu, flb_fp32.cu,
// flb_bf16.cu) and the precision-independent kernels (flb_fft.cu).
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/flb.h"

namespace flb {

// Tracing: every C-ABI call that launches GPU work opens an NVTX range named
// after the call, so a profiler attributes each kernel to the call that issued
// it (e.g. ncu --nvtx --nvtx-include "flb_step/").  NVTX is header-only and
// costs a few nanoseconds per range when no profiler is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define FLB_TRACE() ::flb::NvtxRange flb_trace_range_(__func__)

// Planes of z per thread block of the z-marching kernels unless a context sets
// its own (flb_options.z_chunk, or the length flb_step's tuning picks).
constexpr int kZChunkDefault = 16;

// Model parameters in double; each instantiation converts to its compute type.
struct HostModel {
    int Q, D, X, Y, Z;
    long V;
    double rho0;
    double om_s, om_b, om_g, kT;
    int nonideal;
    double A, B, rho_c, kappa;
    int total;  // psi is the total bulk free energy: F gains cs^2 grad rho
    int model;  // 0 force-based, 1 modified equilibrium (D2Q9)
    const void* swift_xi = nullptr;  // modified equilibrium: FFT of the coloured e/eps noise (double2 or float2)
    uint64_t seed;
    uint32_t replica;
    int noise_local;
    int zchunk = 0;  // z-marching kernels: planes per block (0: the built-in default)
};

// Kernels whose code depends on the compute/storage type.  Pointers are device
// pointers; `pop` buffers hold Q*V elements of the storage type, `field`
// buffers V (or 3V) elements of the compute type.
struct PrecOps {
    int elem_size;    // bytes per stored population
    int real_size;    // bytes per compute-type scalar (density/force fields)
    cudaError_t (*density)(const HostModel&, const void* pop, void* drho, cudaStream_t);
    cudaError_t (*step)(const HostModel&, uint64_t step, const void* src, void* dst, const void* drho,
                        cudaStream_t);
    cudaError_t (*init)(const HostModel&, void* dst, const double* rho, const double* u, int thermal,
                        cudaStream_t);
    cudaError_t (*get_pop)(const HostModel&, const void* src, double* out, cudaStream_t);
    cudaError_t (*set_pop)(const HostModel&, const double* in, void* dst, cudaStream_t);
    // which: 0 rho, 1 u (needs F or NULL for the ideal gas), 2 modes
    cudaError_t (*moments)(const HostModel&, const void* src, double* out, int which, const void* F,
                           cudaStream_t);
    cudaError_t (*mu_force)(const HostModel&, const void* drho, void* mu, void* F, cudaStream_t);
    // per-block partial sums; returns the number of partial rows written
    cudaError_t (*mode_partials)(const HostModel&, const void* src, double* partials, int* nrows,
                                 cudaStream_t);
    cudaError_t (*cons_partials)(const HostModel&, const void* src, double* partials, int* nrows,
                                 cudaStream_t);
    // mode a of the pre-collision state as a complex field: double2, or float2
    // when fp32 (the transform of single-precision states)
    cudaError_t (*mode_field)(const HostModel&, const void* src, int mode, void* out, bool fp32, cudaStream_t);
    int (*partial_rows_max)(const HostModel&);
    int (*step_needs_density)(const HostModel&);
    // pre-collision deviations in the storage type, [i][s], to / from a device buffer
    cudaError_t (*pull_state)(const HostModel&, const void* src, void* out, cudaStream_t);
    cudaError_t (*push_state)(const HostModel&, const void* in, void* dst, cudaStream_t);
    // pre-collision populations f_i at n sites (device list), out[i*n + k]
    cudaError_t (*get_sites)(const HostModel&, const void* src, const long long* sites, int n, double* out,
                             cudaStream_t);
    // the step, also writing *nrows rows of 4 partial sums (mass deviation,
    // momentum) of the state it steps from; cudaErrorNotSupported (nothing
    // launched) where the step kernel does not provide them
    cudaError_t (*step_rows)(const HostModel&, uint64_t step, const void* src, void* dst, const void* drho,
                             double* rows, int* nrows, cudaStream_t);
};

const PrecOps& ops_fp64();
const PrecOps& ops_fp32();
const PrecOps& ops_bf16();

// Deterministic column sums: out[c] = sum_r partials[r*ncol + c], plus add0
// on column 0 (flb_fft.cu).
cudaError_t sum_columns(const double* partials, int nrows, int ncol, double* out, cudaStream_t s,
                        double add0 = 0.0);

// True when an axis of length L is transformed by the in-place mixed-radix FFT
// (L a product of 2, 3 and 5, at most 4096); other lengths need `scratch`.
bool fft_length_in_place(int L);

// Record the calling thread's last error message (flb_last_error) and return code.
int set_error(int code, const std::string& msg);

// In-place forward DFT along every axis of length > 1 of a complex X*Y*Z field
// (FP64, and an FP32 form for fields whose precision needs no more).
cudaError_t fft3d(double2* data, int X, int Y, int Z, double2* scratch, cudaStream_t s);
cudaError_t fft3d(float2* data, int X, int Y, int Z, float2* scratch, cudaStream_t s);
// In-place forward DFT of n consecutive rows of length X (scratch: X n elements).
cudaError_t fft_rows(double2* data, int X, int n, double2* scratch, cudaStream_t s);

// Modified-equilibrium model (flb_swift.cu).  swift_table fills chol with
// (c11, c21, c22) per wavevector, the lower Cholesky factor of the lattice
// covariance of the e and eps noise; false (with a message) where it is not
// positive definite.  swift_noise draws the white e/eps normals of `step`,
// transforms them to Fourier space, colours them with chol and leaves in
// `out` a field whose real part times 1/V is xi_e and minus imaginary part
// times 1/V is xi_eps; `work` is scratch (both V complex numbers, float2 when
// fp32, else double2).
bool swift_table(const HostModel& m, double* chol, std::string& err);
cudaError_t swift_noise(const HostModel& m, uint64_t step, const double* chol, void* work, void* out, bool fp32,
                        cudaStream_t s);

// Interface heights of a stripe (flb_capillary.cu): drho is the density
// deviation field (real_size 4 or 8 bytes), h receives 2 X doubles.
cudaError_t interface_heights(const void* drho, int real_size, double rho0, int X, int Y,
                              const flb_interface_fit& f, double* h, cudaStream_t s);
// Height spectrum of the 2 X heights h: work and scratch hold 2 X complex
// doubles; accumulate: acc += p, else out = p (X doubles).
cudaError_t height_power(const double* h, int X, double2* work, double2* scratch, double* acc, double* out,
                         cudaStream_t s);

// Adjoint of one D3Q19 step (flb_adjoint.cu): gn, lam_next, lam are [19][V]
// pre-collision deviations / adjoints in the storage type (FP64 or FP32);
// work holds 10 V compute-type scalars, rows adjoint_rows(m) * 6 doubles;
// grad (6 doubles, device) is incremented.  Within a segment the
// density part of the adjoint (one scalar per site, added to every
// population) may be passed on instead of added: rb_out (V scalars or NULL)
// receives it and the next step takes it as rb_next (NULL: lam_next is
// complete); adjoint_add_rb adds the last one.
cudaError_t adjoint_step(const HostModel& m, int prec, uint64_t step, const void* gn, const void* lam_next,
                         const void* rb_next, void* lam, void* rb_out, void* work, double* rows, double* grad,
                         cudaStream_t st);
cudaError_t adjoint_add_rb(const HostModel& m, int prec, void* lam, const void* rb, cudaStream_t st);
int adjoint_rows(const HostModel& m);

// p = |data|^2 / V with p(0) = 0; accumulate: acc += p, else out = p.
cudaError_t power_spectrum(const double2* data, long V, double* acc, double* out, cudaStream_t s);
cudaError_t power_spectrum(const float2* data, long V, double* acc, double* out, cudaStream_t s);
// out[s] = a * in[s], s < V
cudaError_t scale_copy(const double* in, double a, long V, double* out, cudaStream_t s);

}  // namespace flb
