/*
 * flb.h -- C ABI of the GB300 fluctuating lattice Boltzmann (FLB) library.
 *
 * The library advances the fluctuating lattice Boltzmann equation of
 * M. Gross, M. E. Cates, F. Varnik and R. Adhikari, "Langevin theory of
 * fluctuations in the discrete Boltzmann equation" (arXiv 1012.3632) on one
 * GPU.  One time step is the moment-space update of Sec. V, Eq. (lbe-mom):
 *
 *   f^LB_i(r + c_i, t+1) = (T^-1)_ia [ m_a - w_a (m_a - m_a^eq)
 *                                      + (1 - w_a/2) m^F_a + xi^LB_a ]
 *
 * with m_a = T_ai f^LB_i (Eq. (moments)), m^eq from the second-order discrete
 * Maxwellian (Eq. (feq)), m^F from the forcing term (Eq. (forcing-term), Guo
 * form), relaxation rates w_a = lambda^LB_a (Sec. V) and Gaussian noise
 * xi^LB_a on every non-conserved mode with the lattice fluctuation-dissipation
 * variance of Eq. (noise-lbe):
 *
 *   < xi^LB_a xi^LB_b > = rho kT (2 - w_a) w_a N_a / cs^2  delta_ab,  cs^2 = 1/3.
 *
 * Optionally the fluid is the force-based non-ideal fluid of Sec. IV.B / App. A:
 * F = -rho grad mu, mu = psi'(rho) - kappa lap rho, with the excess free energy
 * psi(rho) = A (rho - rho_c)^2 / 2 + B (rho - rho_c)^4 / 4 and the isotropic
 * lattice stencils grad phi = 3 sum_i w_i c_i phi(r + c_i),
 * lap phi = 6 sum_i w_i (phi(r + c_i) - phi(r)).
 *
 * Conventions shared by every call:
 *  - Return value: FLB_OK (0) or a negative FLB_E* code; flb_last_error()
 *    gives a message for the calling thread's last failure.  No C++
 *    exception crosses this boundary.
 *  - Lattice dimensions are (X, Y, Z) with Z = 1 for D2Q9; the site index is
 *    s = x + X*(y + Y*z) (x fastest); V = X*Y*Z sites.
 *  - Host arrays passed in or out are owned by the caller and are copied;
 *    the library never keeps a caller pointer.  The library owns all device
 *    memory it allocates (flb_create) and frees it in flb_destroy.
 *  - Populations exchanged with the caller are the paper's pre-collision
 *    f^LB(r, t) (Eq. (f-aux)) as doubles in the layout f[i*V + s] with the
 *    velocity order below.
 *      D2Q9  (App. B, rows 2-3 of Eq. (TD2Q9)):
 *        (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
 *      D3Q19:
 *        (0,0,0) (1,0,0) (-1,0,0) (0,1,0) (0,-1,0) (0,0,1) (0,0,-1)
 *        (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1)
 *        (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
 *  - Moment basis: D2Q9 as printed in App. B (rho, jx, jy, e, pww, pxy, qx,
 *    qy, eps).  D3Q19 (the paper gives none): weighted Gram-Schmidt of
 *    1; cx, cy, cz; c^2; 3cx^2-c^2, cy^2-cz^2; cxcy, cycz, czcx; c^2 c (x3);
 *    (cy^2-cz^2)cx, (cz^2-cx^2)cy, (cx^2-cy^2)cz; c^4; c^2(3cx^2-c^2),
 *    c^2(cy^2-cz^2) -- modes 0-3 conserved, 4 bulk (omega_bulk), 5-9 shear
 *    (omega_shear), 10-18 ghosts (omega_ghost).  D2Q9: 0-2 conserved,
 *    3 bulk, 4-5 shear, 6-8 ghosts.
 *  - Noise: Philox4x32-10 (Salmon et al., SC'11) with key (seed lo, seed hi)
 *    and counter (site, step, call | tag << 8, replica); Box-Muller on words
 *    (0,1) and (2,3) of each call, uniforms (x + 1/2) 2^-32.  Non-conserved
 *    mode k (counted from 0 in basis order) uses normal k%4 of call k/4.
 *    Tag 0 is the collision noise, tag 1 the thermal initial state.  Any
 *    site's noise at any step can be recomputed from (seed, replica, site,
 *    step).
 *  - Every call is enqueued on the context's CUDA stream; calls that return
 *    host data synchronise that stream.  A context must not be used by two
 *    host threads at once.
 */
#ifndef FLB_H
#define FLB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FLB_OK 0
#define FLB_EINVAL (-1)    /* invalid argument (e.g. omega not in (0,2), kT < 0, dims < 1) */
#define FLB_ENOMEM (-2)    /* device or host allocation failed */
#define FLB_ECUDA (-3)     /* a CUDA runtime call failed; see flb_last_error() */
#define FLB_EDIVERGED (-4) /* non-finite mass or momentum detected after a step */
#define FLB_ETIMEOUT (-5)  /* reserved: a bounded device-side wait gave up */
#define FLB_EIO (-6)       /* checkpoint file could not be read or written */
#define FLB_EBOUNDS (-7)   /* a guard zone around a device buffer was overwritten */

typedef struct flb_ctx flb_ctx;

typedef enum { FLB_D2Q9 = 9, FLB_D3Q19 = 19 } flb_lattice;

/* Storage precision of the populations.  FP64: doubles, all arithmetic in
 * double.  FP32: deviations g_i = f_i - w_i rho0 stored and computed in float.
 * BF16: deviations stored as bfloat16, arithmetic in float. */
typedef enum { FLB_FP64 = 0, FLB_FP32 = 1, FLB_BF16 = 2 } flb_precision;

/* Observables of flb_moments. */
typedef enum {
    FLB_RHO = 0,      /* out[V]: rho = sum_i f_i (Eq. (lbe-moments)) */
    FLB_U = 1,        /* out[D*V]: u = (sum_i f_i c_i + F/2) / rho (Eq. (lbe-moments)) */
    FLB_MODES = 2,    /* out[Q*V]: m_a = T_ai f_i (Eq. (moments)) */
    FLB_MODE_VAR = 3  /* out[Q]: adds the current state to the snapshot accumulators and
                         returns the mean over snapshots of (1/V) sum_r (m_a - <m_a>_r)^2 */
} flb_observable;

/* Square-gradient free energy of the non-ideal fluid (App. A, Eq. (freeE-funct)):
 * psi(rho) = A (rho - rho_c)^2 / 2 + B (rho - rho_c)^4 / 4 and the gradient term
 * kappa |grad rho|^2 / 2, mu = psi'(rho) - kappa lap rho.  The force is
 *   total = 0: F = -rho grad mu; psi is the excess over the ideal lattice gas,
 *              whose pressure rho cs^2 the LB supplies itself;
 *   total = 1: F = -rho grad mu + cs^2 grad rho; psi is the total bulk free
 *              energy f0 and F is Eq. (he-force), kappa rho grad lap rho -
 *              grad(p0 - rho cs^2) with grad p0 = rho grad f0' (p0 = rho f0' - f0).
 *              The Landau double well of Sec. VI, beta (rho - rho_V)^2 (rho - rho_L)^2,
 *              is A = -beta (rho_L - rho_V)^2, B = 4 beta, rho_c = (rho_L + rho_V) / 2.
 * Gradients and Laplacians are the isotropic lattice stencils
 * grad phi = (1/cs^2) sum_i w_i c_i phi(r + c_i), lap phi = (2/cs^2) sum_i w_i (phi(r + c_i) - phi(r)).
 * enabled = 0: ideal gas. */
typedef struct {
    int enabled;
    double A, B, rho_c, kappa;
    int total;
    int model;  /* 0: force-based model (App. A, above); 1: modified-equilibrium
                   model (Sec. IV.C), D2Q9 only: no force; the equilibrium carries
                   the pressure p = p0(rho) - kappa rho lap rho in e and eps
                   (Eq. (meq-yeo): e += 6 (p - rho cs^2), eps = -6 (p - rho cs^2)) and
                   the square-gradient stress kappa (d_a rho d_b rho - |grad rho|^2
                   delta_ab / 2) in p_ww and p_xy, with p0 = rho psi' - psi
                   (+ rho cs^2 when total = 0); the e and eps noise is drawn in
                   Fourier space around rho0 (times sqrt(rho / rho0) per site with
                   noise_rho_local) with the k-dependent covariance of Eq. (noise-yeo)
                   (corner 6 (c_s^2(k) - cs^2)(lambda_e + lambda_eps), from the FDT)
                   mapped to the lattice as in Sec. V, c_s^2(k) = dp0/drho(rho0) +
                   kappa rho0 K2(k) with K2 the symbol of -lap; flb_create fails
                   with FLB_EINVAL where that covariance is not positive definite. */
} flb_free_energy;

typedef struct {
    int precision;       /* flb_precision (default FLB_FP32) */
    double rho0;         /* reference density of the deviation storage (default 1) */
    uint32_t replica;    /* fourth Philox counter word (default 0) */
    int noise_rho_local; /* 1 (default): local pre-collision rho in the noise variance
                            (Sec. VI, local values in inhomogeneous states); 0: rho0 */
    void* stream;        /* cudaStream_t to enqueue on; NULL: the legacy default stream */
    int device;          /* CUDA device ordinal; -1 (default): the current device */
    int check_every;     /* flb_step checks mass/momentum for NaN/Inf every this many
                            steps (0: never; default 0) */
    int guard;           /* 1: the two population buffers and the density field get
                            64 KiB guard zones of a fixed byte pattern on both sides,
                            checked by flb_check_guards (a bounds check of the
                            kernels' writes for debugging; default 0) */
    int z_chunk;         /* D3Q19 non-ideal step (z-marching kernels): planes of z per
                            thread block.  0 (default): flb_step times candidate
                            lengths on its first steps (three launches each, CUDA
                            events, one host wait on them when done) and keeps
                            the fastest; > 0: that length (at most Z).  The chunk
                            length changes no result: every site's arithmetic is
                            the same. */
} flb_options;

/* Fill *opt with the defaults listed above. */
void flb_default_options(flb_options* opt);

/* Create a context for a periodic lattice and allocate its device state.
 *   lattice  FLB_D2Q9 or FLB_D3Q19
 *   dims     (X, Y, Z), each >= 1; Z must be 1 for D2Q9; X*Y*Z < 2^31
 *   omega_*  lattice relaxation rates lambda^LB (Sec. V) of the shear, bulk and
 *            ghost modes, each in (0, 2)
 *   kT       noise temperature >= 0 (kT = 0: deterministic MRT-LB)
 *   fe       free energy (NULL or enabled = 0: ideal gas)
 *   seed     64-bit Philox key
 *   opt      NULL for defaults
 * The state is the uniform rest state f = w rho0 at step 0.  Returns
 * FLB_EINVAL for bad arguments (context not created), FLB_ENOMEM, FLB_ECUDA. */
int flb_create(flb_ctx** out, int lattice, const int dims[3], double omega_shear,
               double omega_bulk, double omega_ghost, double kT, const flb_free_energy* fe,
               uint64_t seed, const flb_options* opt);

/* Set the state to f^eq(rho, u) (Eq. (feq)); with thermal_init != 0 every mode a
 * (conserved ones included) additionally receives a Gaussian of variance
 * rho kT N_a / cs^2, the ideal-gas equal-time variance of Eqs. (G-ideal) and
 * (mu-ideal) (noise tag 1, step 0).  rho: host array of V doubles or NULL (rho0);
 * u: host array of D*V doubles (u[d*V + s]) or NULL (rest).  Resets the step
 * counter to 0 and clears the accumulators. */
int flb_init(flb_ctx* ctx, const double* rho, const double* u, int thermal_init);

/* Advance nsteps >= 0 time steps (Eq. (lbe-mom) + streaming, periodic).  With
 * check_every > 0, returns FLB_EDIVERGED when the total mass or momentum is no
 * longer finite. */
int flb_step(flb_ctx* ctx, int nsteps);

/* Copy an observable of the current pre-collision state into the host array
 * out (size given with flb_observable).  Synchronises the stream. */
int flb_moments(flb_ctx* ctx, double* out, int which);

/* Structure factor of mode `mode` (0 = density, giving G_11(k) = S(k) of
 * Sec. IV, Eq. (g-correl)): S_a(k) = |sum_r dm_a(r) exp(-i k.r)|^2 / V with
 * dm_a = m_a - <m_a>_r and k = 2 pi (n_x/X, n_y/Y, n_z/Z), computed by an FFT in
 * double precision; S_a(0) = 0.  With accumulate != 0 the snapshot is added to
 * the mode's double-precision accumulator and S (host, V doubles indexed like
 * sites by (n_x, n_y, n_z); may be NULL) receives the mean over all accumulated
 * snapshots of the mode; with accumulate = 0, S receives the current snapshot
 * and the accumulator is untouched. */
int flb_structure_factor(flb_ctx* ctx, double* S, int mode, int accumulate);

/* Number of snapshots accumulated for structure factors of `mode`
 * (mode = -1: the FLB_MODE_VAR accumulators; mode = -2: flb_height_spectrum). */
int flb_snapshot_count(flb_ctx* ctx, int mode, int* count);

/* Clear every snapshot accumulator. */
int flb_reset_accumulators(flb_ctx* ctx);

/* ---- Capillary fluctuations of a liquid stripe (Sec. VI) ------------------
 * A 2-D (D2Q9) state holding a liquid stripe between two interfaces normal to
 * y: the lower one (vapour below, liquid above) near row guess[0], the upper
 * one (liquid below, vapour above) near row guess[1]. */
typedef struct {
    double rho_l, rho_v; /* liquid and vapour density of the fitted profile */
    double width;        /* interface width w of Eq. (interf-width), > 0 */
    double guess[2];     /* rows of the lower and the upper interface */
    int window;          /* rows fitted on each side of round(guess[i]); >= 1, 2 window + 1 <= Y */
    int iterations;      /* Gauss-Newton iterations from h = guess[i]; 1..100 */
} flb_interface_fit;

/* Heights of the two interfaces in every column (Eq. (height-def)): for each
 * column x and interface i, h minimizes
 *   sum over rows y = c - window .. c + window (c = round(guess[i]), periodic)
 *   of (rho(x, y) - rho_MF(y - h))^2,
 *   rho_MF(s) = (rho_l + rho_v)/2 +- (rho_l - rho_v)/2 tanh(2 s / width)
 * (the mean-field profile of Eq. (denprof); + for the lower interface), by
 * `iterations` Gauss-Newton steps from h = guess[i].  rho is the pre-collision
 * density of the current state.  h: host, 2 X doubles (lower interface first,
 * caller-owned).  FLB_EINVAL for a D3Q19 context or invalid fit parameters. */
int flb_interface_heights(flb_ctx* ctx, const flb_interface_fit* fit, double* h);

/* Height spectrum of the two interfaces, averaged over both:
 *   S(k_n) = (1/2) sum_i |sum_x (h_i(x) - <h_i>) e^{-2 pi i n x / X}|^2 / X,
 * n = 0 .. X-1 (S(0) = 0), the quantity Eq. (capill-static) compares with
 * kT / (sigma (2 - 2 cos k)) on the lattice.  accumulate = 1 adds the current
 * state to the running sum (count: flb_snapshot_count with mode -2) and S
 * receives the mean over the snapshots; accumulate = 0 returns the current
 * state's spectrum.  S: host, X doubles, or NULL.  Errors as
 * flb_interface_heights; device memory (a few X doubles) is allocated on the
 * first call. */
int flb_height_spectrum(flb_ctx* ctx, const flb_interface_fit* fit, double* S, int accumulate);

/* Planes of z per thread block of the D3Q19 non-ideal step (opt.z_chunk):
 * *planes = the length in use (the built-in default while tuning or for other
 * steps), *tuning = 1 while flb_step is still timing candidates. */
int flb_z_chunk(flb_ctx* ctx, int* planes, int* tuning);

/* Bounds check of the kernels' writes (contexts created with opt.guard = 1):
 * waits for the context's stream, copies every guard zone to the host and
 * returns FLB_OK when each still holds its pattern, FLB_EBOUNDS when one was
 * overwritten (flb_last_error names the buffer, the side and the first changed
 * byte), FLB_EINVAL when the context has no guard zones.  Reads outside a
 * buffer are not detected. */
int flb_check_guards(flb_ctx* ctx);

/* flb_step(ctx, nsteps) that also reports, for every step, the total mass and
 * momentum of the state the step starts from: sums[4*t + 0] = sum rho,
 * sums[4*t + 1..3] = sum_r sum_i f_i c_i (as flb_conservation), t < nsteps.
 * sums: host, 4*nsteps doubles, written when the call returns (it waits for
 * the context's stream once, at the end; device-addressable page-locked
 * memory is written in place by the reduction, other memory through a copy).  The D3Q19 force-model step with
 * FP32 or BF16 storage and even X forms these sums inside the step kernel
 * (per-block partial sums of the mass deviation and momentum its collision
 * forms from the pulled populations); every other step runs the reduction of
 * flb_conservation before the step.  Errors as flb_step. */
int flb_step_sums(flb_ctx* ctx, int nsteps, double* sums);

/* flb_step_sums without the wait: enqueues the nsteps steps and the delivery
 * of their sums (the same 4*nsteps doubles, mass included) into the host
 * array sums on the context's stream and returns.  sums must stay valid and
 * unread until the stream has been synchronised (flb_synchronize, or any call
 * that waits for the stream).  Page-locked host memory that the device can
 * address (cudaHostAlloc / cudaMallocHost, or registered, under unified
 * addressing) receives the sums straight from the reduction kernel; other
 * memory gets them by a copy from device rows on the stream (asynchronous for
 * page-locked memory; with pageable memory the runtime may wait for it), and
 * a later call reuses those rows only after this call's copy in stream order.
 * Errors as flb_step (a failed launch is reported by this call, a failure
 * inside a kernel by the next synchronising call). */
int flb_step_sums_async(flb_ctx* ctx, int nsteps, double* sums);

/* Total mass and momentum of the current state, summed on the GPU in double:
 * out[0] = sum rho, out[1..3] = sum_r sum_i f_i c_i (z component 0 for D2Q9). */
int flb_conservation(flb_ctx* ctx, double out[4]);

/* Read / write the pre-collision populations f^LB (host, Q*V doubles). */
int flb_get_populations(flb_ctx* ctx, double* f);
int flb_set_populations(flb_ctx* ctx, const double* f);

/* Pre-collision populations f^LB at n chosen sites, without copying the
 * lattice (sampling large lattices).  sites: host, n site indices
 * x + X*(y + Y*z), each in [0, V) (else FLB_EINVAL before any GPU work; n = 0
 * does nothing).  f: host, Q*n doubles, f[i*n + k] = f_i at sites[k], the same
 * values as flb_get_populations' f[i*V + sites[k]].  Device memory for the
 * list and the result is allocated and freed inside the call. */
int flb_get_sites(flb_ctx* ctx, const long long* sites, int n, double* f);

/* ---- Adjoint -----------------------------------------------------------------
 * Device-side state exchange and the adjoint (reverse-mode derivative) of one
 * D3Q19 time step, for gradient-based use (e.g. behind an autograd function
 * with checkpointing).  The paper derives no adjoint; the step differentiated
 * is exactly the forward update of flb_step (Eq. (lbe-mom), the force model of
 * App. A and the noise with its local-density amplitude, replayed from the
 * same Philox counters).
 *
 * State buffers are caller-owned device arrays of 19*V elements of the storage
 * type (double for FLB_FP64, float for FLB_FP32) holding pre-collision
 * deviations g_i = f_i - w_i rho0 in the layout g[i*V + s]. */

/* Copy the current state into g (enqueued, no synchronisation). */
int flb_get_state_device(flb_ctx* ctx, void* g);
/* Replace the current state by g (enqueued, no synchronisation). */
int flb_set_state_device(flb_ctx* ctx, const void* g);

/* Given the state g_n at time `step` and lam_next = dJ/dg at time step+1,
 * write lam = dJ/dg at time `step` (must not alias lam_next) and add to the
 * device array grad[6] the derivatives dJ/d(omega_shear, omega_bulk,
 * omega_ghost, kappa, A, B) contributed by this step.  D3Q19, FP64 or FP32
 * contexts only (FLB_EINVAL otherwise).  Work arrays are allocated on first
 * use.  Enqueued on the context's stream. */
int flb_adjoint_step(flb_ctx* ctx, const void* g_n, uint64_t step, const void* lam_next, void* lam, double* grad);

/* One checkpoint segment of the reverse pass in a single call.  From the
 * state g_start at time step0, recompute the states at step0 .. step0+n-1
 * (n >= 1) into `states`, a caller-owned device array of n*19*V elements of
 * the storage type (states[k*19*V + i*V + s]), then apply flb_adjoint_step
 * from time step0+n-1 down to step0.  lam: device, 19*V elements, holds
 * dJ/dg at time step0+n on entry and dJ/dg at time step0 on return; grad[6]
 * accumulates as in flb_adjoint_step.  The recomputation runs the context's
 * own step (its state and step counter end at time step0+n-1).  Errors and
 * restrictions as flb_adjoint_step; enqueued on the context's stream. */
int flb_adjoint_segment(flb_ctx* ctx, const void* g_start, uint64_t step0, int n, void* states, void* lam,
                        double* grad);

/* Step counter (the time index keying the collision noise). */
int flb_get_step(flb_ctx* ctx, uint64_t* step);
int flb_set_step(flb_ctx* ctx, uint64_t step);

/* Enqueue subsequent work on another cudaStream_t (NULL: legacy default stream). */
int flb_set_stream(flb_ctx* ctx, void* stream);

/* Wait for the context's stream. */
int flb_synchronize(flb_ctx* ctx);

/* Query sizes: out[0] = Q, out[1] = D, out[2..4] = X, Y, Z, out[5] = precision. */
int flb_get_info(flb_ctx* ctx, int out[6]);

/* Per-kernel CUDA-event timing of flb_step (off by default).  While enabled,
 * every kernel that flb_step launches is bracketed by events on the context's
 * stream.  flb_kernel_times fills ms[k] (total milliseconds) and launches[k]
 * for k < FLB_NKERNEL_TIMERS: 0 = density gather, 1 = fused stream-collide,
 * 2 = conservation check.  Enabling or disabling clears the totals. */
#define FLB_NKERNEL_TIMERS 3
int flb_kernel_timing(flb_ctx* ctx, int enable);
int flb_kernel_times(flb_ctx* ctx, double* ms, int* launches);

/* ---- Batched replicas -------------------------------------------------------
 * Up to FLB_BATCH_MAX independent periodic D3Q19 ideal-gas lattices of uneven
 * sizes, advanced together for ensemble averages (the equilibration-ratio
 * statistics of Sec. VI).  Each time step is one persistent kernel launch over
 * the flattened (replica, tile) work list; steps are replayed from a captured
 * CUDA graph of two steps.  Populations are FP32 deviations.  Replica r uses
 * the Philox key seeds[r] and counter word replica = opt->replica + r, so its
 * noise is that of a single context created with the same seed and replica
 * word.  Observables are per replica. */
#define FLB_BATCH_MAX 96
typedef struct flb_batch flb_batch;

/* n replicas; dims: n*3 ints; omega_shear, kT, seeds: n values; omega_bulk and
 * omega_ghost: n values or NULL (1.0).  opt: precision must be FLB_FP32 (the
 * default); rho0, replica, noise_rho_local, stream and device as for
 * flb_create.  State: rest at step 0.  FLB_EINVAL for bad arguments. */
int flb_batch_create(flb_batch** out, int lattice, int n, const int* dims, const double* omega_shear,
                     const double* omega_bulk, const double* omega_ghost, const double* kT,
                     const uint64_t* seeds, const flb_options* opt);

/* Rest state f = w rho0 in every replica, plus the thermal modes of flb_init
 * when thermal_init != 0; resets the step counter and the accumulators. */
int flb_batch_init(flb_batch* b, int thermal_init);

/* Advance every replica nsteps time steps (graph replays of two steps). */
int flb_batch_step(flb_batch* b, int nsteps);

/* Time each candidate tile shape (x, y, z; 256 sites, powers of two) on the
 * replicas of each distinct lattice size and keep the fastest per size; the
 * state is not advanced.  shapes (n*3 ints, may be NULL) receives the choice. */
int flb_batch_autotune(flb_batch* b, int* shapes);

/* Add the current state to the per-replica snapshot accumulators and return in
 * out[r*19 + a] the mean over snapshots of (1/V_r) sum (m_a - <m_a>)^2. */
int flb_batch_mode_variance(flb_batch* b, double* out);

/* Structure factor of one replica, as flb_structure_factor. */
int flb_batch_structure_factor(flb_batch* b, int replica, double* S, int mode, int accumulate);

/* Pre-collision populations of one replica (host, 19*V_r doubles). */
int flb_batch_get_populations(flb_batch* b, int replica, double* f);

/* Number of replicas, total sites, step counter (each may be NULL). */
int flb_batch_info(flb_batch* b, int* n, long long* sites, uint64_t* step);

int flb_batch_synchronize(flb_batch* b);
void flb_batch_destroy(flb_batch* b);

/* Structure factor that allocates nothing.  For callers that cannot allocate
 * device memory while they run -- hosts whose allocator forbids cudaMalloc
 * after start-up (a serving process that sizes its device memory once),
 * real-time loops with a fixed memory budget, code running where an
 * allocation would synchronise the device -- this computes, from buffers the
 * caller already owns, the same S_a(k) as flb_structure_factor
 * (accumulate = 0).  The paper has no counterpart: it is an interface variant
 * of flb_structure_factor.
 *   lattice  FLB_D2Q9 or FLB_D3Q19;  dims as in flb_create, every edge a
 *            product of 2, 3 and 5 (up to 4096) and at most
 *            FLB_NOALLOC_MAX_SITES sites in all; anything else returns
 *            FLB_EINVAL before any GPU work
 *   f        device pointer: pre-collision populations f^LB, Q*V doubles in the
 *            layout f[i*V + s] (what flb_get_populations returns), read only
 *   mode     0 = density, else the mode index of the basis above
 *   S        device pointer to V doubles, overwritten with S_a(k) (S_a(0) = 0)
 *   stream   cudaStream_t to enqueue on (NULL: legacy default stream); the
 *            call returns after enqueueing, without synchronising
 * The FFT work array is a static device array of FLB_NOALLOC_MAX_SITES complex
 * doubles (16 MiB) that every GPU which loads the library holds until the
 * process exits.  The first call on a device sets that device up: with the
 * device current it looks up the array's device address
 * (cudaGetSymbolAddress), reads the SM count and raises the FFT kernel's
 * shared-memory limit (host-side runtime calls; none of them allocates).  The
 * look-up is kept for the life of the process: after a cudaDeviceReset in the
 * caller's process this entry point must not be called again.  Every call
 * uses the same array, which keeps the last call's contents (each call
 * overwrites all of the part it reads), so calls that may overlap on the GPU
 * (unordered streams, several host threads) race and must be serialised by the
 * caller.  No cudaMalloc, cudaFree or allocating library routine is called. */
#define FLB_NOALLOC_MAX_SITES (1 << 20)
int flb_structure_factor_noalloc(int lattice, const int dims[3], const double* f, int mode, double* S,
                                 void* stream);

/* Checkpoint: parameters, step counter, seed, replica and the populations in
 * the stored precision; a resumed run continues bit for bit. */
int flb_save(flb_ctx* ctx, const char* path);
int flb_load(flb_ctx** out, const char* path, const flb_options* opt);

/* Message for an error code / for the calling thread's last failure. */
const char* flb_error_string(int code);
const char* flb_last_error(void);

/* Free the context and all its device memory (NULL is ignored). */
void flb_destroy(flb_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* FLB_H */
