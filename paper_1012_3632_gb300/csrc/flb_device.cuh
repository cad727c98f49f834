// flb_device.cuh -- device building blocks of the fluctuating lattice Boltzmann
// step: counter-based normals, the hand-derived moment transforms of D2Q9 and
// D3Q19, and the moment-space collision of Gross, Cates, Varnik & Adhikari
// (arXiv 1012.3632), Sec. V, Eq. (lbe-mom), with the lattice FDT noise of
// Eq. (noise-lbe).
//
// Populations are handled as deviations g_i = f_i - w_i rho0 from the rest
// state.  Every non-conserved moment of w_i rho0 vanishes (weighted
// orthogonality, Eq. (T-orthog)), so only the density moment shifts:
// rho = rho0 + sum_i g_i.
//
// The transforms are written out by hand, pairing each velocity c with -c:
// even moments use s = g(c) + g(-c), odd moments d = g(c) - g(-c).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_bf16.h>

namespace flb {

// ---------------------------------------------------------------------------
// Storage conversions
// ---------------------------------------------------------------------------
template <class R, class S>
__device__ __forceinline__ R load_s(const S* p) { return static_cast<R>(*p); }
template <>
__device__ __forceinline__ float load_s<float, __nv_bfloat16>(const __nv_bfloat16* p)
{
    return __bfloat162float(*p);
}
template <class R, class S>
__device__ __forceinline__ void store_s(S* p, R v) { *p = static_cast<S>(v); }
template <>
__device__ __forceinline__ void store_s<float, __nv_bfloat16>(__nv_bfloat16* p, float v)
{
    *p = __float2bfloat16_rn(v);
}

// Streaming variants for the time step: a stored population is not read again
// before the next step, and the last read of a population within a step need
// not stay in L2 (evict-first / last-use hints keep L2 for data still to be
// re-read).
template <class R, class S>
__device__ __forceinline__ void store_stream(S* p, R v) { __stcs(p, static_cast<S>(v)); }
template <>
__device__ __forceinline__ void store_stream<float, __nv_bfloat16>(__nv_bfloat16* p, float v)
{
    __stcs(reinterpret_cast<unsigned short*>(p), __bfloat16_as_ushort(__float2bfloat16_rn(v)));
}
template <class R, class S>
__device__ __forceinline__ R load_last(const S* p) { return static_cast<R>(__ldlu(p)); }
template <>
__device__ __forceinline__ float load_last<float, __nv_bfloat16>(const __nv_bfloat16* p)
{
    return __bfloat162float(__ushort_as_bfloat16(__ldlu(reinterpret_cast<const unsigned short*>(p))));
}

// ---------------------------------------------------------------------------
// Counter-based random numbers
// ---------------------------------------------------------------------------

// Philox key schedule: the round keys k0 + r W0, k1 + r W1 (r = 0..9), computed
// once on the host so that each round reads them from the parameter bank.
struct PhiloxKeys {
    uint32_t k[20];  // k[r] = k0 + r W0, k[10 + r] = k1 + r W1
};

inline PhiloxKeys philox_keys(uint64_t seed)
{
    PhiloxKeys K;
    uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.k[r] = k0;
        K.k[10 + r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return K;
}

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& K)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32x32 -> 64-bit multiply per word pair gives both halves
        const unsigned long long p0 = 0xD2511F53ull * c.x;
        const unsigned long long p1 = 0xCD9E8D57ull * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ K.k[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ K.k[10 + r],
                       (uint32_t)p0);
    }
    return c;
}

// One round of philox4x32_10 with round keys k0, k1 (for callers that run
// several counters' rounds in lock-step).
__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t k0, uint32_t k1)
{
    const unsigned long long p0 = 0xD2511F53ull * c.x;
    const unsigned long long p1 = 0xCD9E8D57ull * c.z;
    return make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
}

// SFU approximations (PTX lg2/rsqrt/rcp/sin/cos .approx.ftz.f32).  Their
// arguments here are normal numbers, for which the flush-to-zero forms give
// the same results; they skip the handling of subnormal operands, which took
// a third of the Box-Muller transform's instructions.
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_approx(float x)
{
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_approx(float x)
{
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Box-Muller on a pair of 32-bit words; uniforms (x + 1/2) 2^-32 lie in (0, 1].
// Single precision on the SFU: -2 ln u0 = (-2 ln 2) log2 u0, the radius via
// rsqrt, and cos/sin(2 pi u) = -cos/-sin(2 pi u - pi) with the argument in
// [-pi, pi], where the approximate sine and cosine are accurate to about
// 2^-21 absolute.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1)
{
    const float u0 = fmaf(__uint2float_rn(a), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    const float u1 = fmaf(__uint2float_rn(b), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    const float t = fmaxf(-1.3862943611198906f * lg2_approx(u0), 1e-30f);  // u0 may round to 1: radius 0, not NaN
    const float r = t * rsqrt_approx(t);
    const float w = fmaf(u1, 6.28318530717958648f, -3.14159265358979324f);
    z0 = -r * cos_approx(w);
    z1 = -r * sin_approx(w);
}
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double& z0, double& z1)
{
    const double u0 = ((double)a + 0.5) * 2.3283064365386963e-10;
    const double u1 = ((double)b + 0.5) * 2.3283064365386963e-10;
    const double r = sqrt(-2.0 * log(u0));
    double s, c;
    sincospi(2.0 * u1, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// Four standard normals from the call (site, step, call | tag << 8, replica).
template <class R>
__device__ __forceinline__ void normals4(const PhiloxKeys& K, uint32_t site, uint32_t step, uint32_t call_tag,
                                         uint32_t replica, R z[4])
{
    const uint4 r = philox4x32_10(make_uint4(site, step, call_tag, replica), K);
    box_muller(r.x, r.y, z[0], z[1]);
    box_muller(r.z, r.w, z[2], z[3]);
}

// ---------------------------------------------------------------------------
// Collision parameters (per launch, in the kernel's parameter bank)
// ---------------------------------------------------------------------------
// Per non-conserved mode k (mode a = D + 1 + k) the kernel adds
//   (m*_a - m_a) / N_a = frc[k] m^F_a + rel[k] (m_a - m^eq_a) + ns[k] sqrt(rho) z_k
// with rel = -omega_a / N_a, frc = (1 - omega_a / 2) / N_a (stress modes only; the
// ghosts have m^eq = m^F = 0) and ns = sqrt(kT omega_a (2 - omega_a) N_a / cs^2) / N_a.
template <class R>
struct Coll {
    R rho0, sqrt_rho0;
    R rel[16];
    R frc[6];
    R ns[16];
    int noise;            // kT > 0
    int noise_local;      // local rho (1) or rho0 (0) in the noise variance
    PhiloxKeys key;       // Philox round keys
    uint32_t step;        // time step keying the noise (single-lattice launches)
    uint32_t replica;     // fourth Philox counter word
};

// ---------------------------------------------------------------------------
// Two lattice sites in one register pair: packed single-precision arithmetic
// (FADD2 / FMUL2 / FFMA2 of sm_100 and later) for kernels that update sites
// x and x+1 together.
// ---------------------------------------------------------------------------
struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit F2(double c) : v(make_float2((float)c, (float)c)) {}
    __device__ __forceinline__ explicit F2(float c) : v(make_float2(c, c)) {}
    __device__ __forceinline__ explicit F2(int c) : v(make_float2((float)c, (float)c)) {}
};
__device__ __forceinline__ F2 mk2(float2 v)
{
    F2 r;
    r.v = v;
    return r;
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return mk2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return mk2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return mk2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator*(float a, F2 b) { return mk2(__fmul2_rn(make_float2(a, a), b.v)); }
__device__ __forceinline__ F2 operator*(F2 a, float b) { return mk2(__fmul2_rn(a.v, make_float2(b, b))); }
__device__ __forceinline__ F2 operator+(float a, F2 b) { return mk2(__fadd2_rn(make_float2(a, a), b.v)); }
__device__ __forceinline__ F2 operator+(F2 a, float b) { return mk2(__fadd2_rn(a.v, make_float2(b, b))); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b)
{
    a = a + b;
    return a;
}
__device__ __forceinline__ F2& operator*=(F2& a, F2 b)
{
    a = a * b;
    return a;
}

// reciprocal and square root: the FP32 paths use the SFU approximations (the
// density is ~1 and the results feed terms far below FP32 storage rounding)
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_(float x) { return rcp_approx(x); }
__device__ __forceinline__ F2 rcp_(F2 x) { return F2(rcp_approx(x.v.x), rcp_approx(x.v.y)); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return x * rsqrt_approx(x); }
__device__ __forceinline__ F2 sqrt_(F2 x) { return F2(sqrt_(x.v.x), sqrt_(x.v.y)); }

// Normals 0..N-1 of the collision noise of `site` (one site per lane).
template <int NCALL, class R>
__device__ __forceinline__ void noise_normals(const PhiloxKeys& K, uint32_t site, uint32_t step, uint32_t rep,
                                              R z[4 * NCALL])
{
#pragma unroll
    for (int b = 0; b < NCALL; ++b) normals4(K, site, step, (uint32_t)b, rep, z + 4 * b);
}
// Box-Muller of two sites at once: the word pairs (a0, a1) of site x and
// (b0, b1) of site x+1, the same arithmetic as box_muller with the FP32 steps
// in packed form (bitwise the same normals; the SFU steps stay per element).
__device__ __forceinline__ void box_muller2(uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1, F2& z0, F2& z1)
{
    const float2 sc = make_float2(2.3283064365386963e-10f, 2.3283064365386963e-10f);
    const float2 of = make_float2(1.1641532182693481e-10f, 1.1641532182693481e-10f);
    const float2 u0 = __ffma2_rn(make_float2(__uint2float_rn(a0), __uint2float_rn(b0)), sc, of);
    const float2 u1 = __ffma2_rn(make_float2(__uint2float_rn(a1), __uint2float_rn(b1)), sc, of);
    const float2 l = __fmul2_rn(make_float2(-1.3862943611198906f, -1.3862943611198906f),
                                make_float2(lg2_approx(u0.x), lg2_approx(u0.y)));
    const float2 t = make_float2(fmaxf(l.x, 1e-30f), fmaxf(l.y, 1e-30f));
    const float2 r = __fmul2_rn(t, make_float2(rsqrt_approx(t.x), rsqrt_approx(t.y)));
    const float2 w = __ffma2_rn(u1, make_float2(6.28318530717958648f, 6.28318530717958648f),
                                make_float2(-3.14159265358979324f, -3.14159265358979324f));
    const float2 nr = make_float2(-r.x, -r.y);
    z0 = mk2(__fmul2_rn(nr, make_float2(cos_approx(w.x), cos_approx(w.y))));
    z1 = mk2(__fmul2_rn(nr, make_float2(sin_approx(w.x), sin_approx(w.y))));
}
// The normals of the two sites (site, site + 1) of a thread: site's in .x,
// site + 1's in .y.  INTERLEAVED: the rounds of all 2 NCALL Philox calls in
// lock-step (round-major) rather than one call after another -- the same
// numbers; which order schedules better depends on the kernel around it.
template <int NCALL, bool INTERLEAVED = false>
__device__ __forceinline__ void noise_normals(const PhiloxKeys& K, uint32_t site, uint32_t step, uint32_t rep,
                                              F2 z[4 * NCALL])
{
    if constexpr (INTERLEAVED) {
        uint4 ca[NCALL], cb[NCALL];
#pragma unroll
        for (int b = 0; b < NCALL; ++b) {
            ca[b] = make_uint4(site, step, (uint32_t)b, rep);
            cb[b] = make_uint4(site + 1, step, (uint32_t)b, rep);
        }
#pragma unroll
        for (int r = 0; r < 10; ++r) {
#pragma unroll
            for (int b = 0; b < NCALL; ++b) {
                ca[b] = philox_round(ca[b], K.k[r], K.k[10 + r]);
                cb[b] = philox_round(cb[b], K.k[r], K.k[10 + r]);
            }
        }
#pragma unroll
        for (int b = 0; b < NCALL; ++b) {
            box_muller2(ca[b].x, ca[b].y, cb[b].x, cb[b].y, z[4 * b], z[4 * b + 1]);
            box_muller2(ca[b].z, ca[b].w, cb[b].z, cb[b].w, z[4 * b + 2], z[4 * b + 3]);
        }
    } else {
#pragma unroll
        for (int b = 0; b < NCALL; ++b) {
            const uint4 ra = philox4x32_10(make_uint4(site, step, (uint32_t)b, rep), K);
            const uint4 rb = philox4x32_10(make_uint4(site + 1, step, (uint32_t)b, rep), K);
            box_muller2(ra.x, ra.y, rb.x, rb.y, z[4 * b], z[4 * b + 1]);
            box_muller2(ra.z, ra.w, rb.z, rb.w, z[4 * b + 2], z[4 * b + 3]);
        }
    }
}

// ---------------------------------------------------------------------------
// D2Q9 (App. B).  Velocity order: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1)
// (-1,-1) (1,-1).  Pairs (c, -c): (1,3) (2,4) (5,7) (8,6).
// Modes: rho, jx, jy, e = 3c^2-2, pww = cx^2-cy^2, pxy = cxcy,
// qx = (3c^2-4)cx, qy = (3c^2-4)cy, eps = 9c^4-15c^2+2;
// N = 1, 1/3, 1/3, 4, 4/9, 1/9, 2/3, 2/3, 16.
// ---------------------------------------------------------------------------
struct D2Q9 {
    static constexpr int Q = 9, D = 2, NNC = 6, NCALL = 2, NCALL_ALL = 3;

    // All nine moments of deviations g (m[0] = sum g).
    template <class R>
    __device__ __forceinline__ static void moments(const R g[9], R m[9])
    {
        const R s1 = g[1] + g[3], d1 = g[1] - g[3];
        const R s2 = g[2] + g[4], d2 = g[2] - g[4];
        const R s3 = g[5] + g[7], d3 = g[5] - g[7];
        const R s4 = g[8] + g[6], d4 = g[8] - g[6];
        const R sa = s1 + s2, sd = s3 + s4;
        m[0] = g[0] + sa + sd;
        m[1] = d1 + d3 + d4;
        m[2] = d2 + d3 - d4;
        m[3] = sa + R(4) * sd - R(2) * g[0];
        m[4] = s1 - s2;
        m[5] = s3 - s4;
        m[6] = R(2) * (d3 + d4) - d1;
        m[7] = R(2) * (d3 - d4) - d2;
        m[8] = R(2) * g[0] - R(4) * sa + R(8) * sd;
    }

    // g_i += w_i sum_a T_ai D_a for the modes a >= 1 (D_a = increment / N_a).
    template <class R>
    __device__ __forceinline__ static void add_back(const R Dm[9], R g[9])
    {
        const R De = Dm[3], Dw = Dm[4], Dxy = Dm[5], Dqx = Dm[6], Dqy = Dm[7], Dep = Dm[8];
        g[0] += R(4.0 / 9.0) * (R(2) * (Dep - De));
        const R E1 = De + Dw - R(4) * Dep, O1 = Dm[1] - Dqx;
        const R E2 = De - Dw - R(4) * Dep, O2 = Dm[2] - Dqy;
        const R E3 = R(4) * De + Dxy + R(8) * Dep, O3 = Dm[1] + Dm[2] + R(2) * (Dqx + Dqy);
        const R E4 = R(4) * De - Dxy + R(8) * Dep, O4 = Dm[1] - Dm[2] + R(2) * (Dqx - Dqy);
        g[1] += R(1.0 / 9.0) * (E1 + O1);
        g[3] += R(1.0 / 9.0) * (E1 - O1);
        g[2] += R(1.0 / 9.0) * (E2 + O2);
        g[4] += R(1.0 / 9.0) * (E2 - O2);
        g[5] += R(1.0 / 36.0) * (E3 + O3);
        g[7] += R(1.0 / 36.0) * (E3 - O3);
        g[8] += R(1.0 / 36.0) * (E4 + O4);
        g[6] += R(1.0 / 36.0) * (E4 - O4);
    }

    // Populations w_i sum_a T_ai D_a of all modes (D_0 included), into g.
    template <class R>
    __device__ __forceinline__ static void from_moments(const R Dm[9], R g[9])
    {
        for (int i = 0; i < 9; ++i) g[i] = R(0);
        add_back(Dm, g);
        g[0] += R(4.0 / 9.0) * Dm[0];
        for (int i = 1; i < 5; ++i) g[i] += R(1.0 / 9.0) * Dm[0];
        for (int i = 5; i < 9; ++i) g[i] += R(1.0 / 36.0) * Dm[0];
    }

    __host__ __device__ static constexpr double N(int a)
    {
        return a == 0 ? 1.0 : a < 3 ? 1.0 / 3 : a == 3 ? 4.0 : a == 4 ? 4.0 / 9 : a == 5 ? 1.0 / 9 : a < 8 ? 2.0 / 3 : 16.0;
    }

    // Moments of f^eq(rho, u) - w rho0 (Eq. (feq); m^eq column of Table I).
    template <class R>
    __device__ __forceinline__ static void eq_moments(R drho, R rho, R ux, R uy, R, R m[9])
    {
        m[0] = drho;
        m[1] = rho * ux;
        m[2] = rho * uy;
        m[3] = R(3) * rho * (ux * ux + uy * uy);
        m[4] = rho * (ux * ux - uy * uy);
        m[5] = rho * ux * uy;
        m[6] = m[7] = m[8] = R(0);
    }

    // Equilibrium (Eq. (feq)) and forcing (Guo form) moments of the stress modes.
    template <class R, class PR>
    __device__ __forceinline__ static void collide(R g[9], R Fx, R Fy, const Coll<PR>& P, uint32_t site,
                                                   uint32_t step)
    {
        R m[9];
        moments(g, m);
        const R rho = P.rho0 + m[0];
        const R ir = rcp_(rho);
        const R ux = (m[1] + R(0.5) * Fx) * ir, uy = (m[2] + R(0.5) * Fy) * ir;
        const R uxx = ux * ux, uyy = uy * uy;
        const R eq_e = R(3) * rho * (uxx + uyy);
        const R eq_w = rho * (uxx - uyy);
        const R eq_xy = rho * ux * uy;
        const R F_e = R(6) * (ux * Fx + uy * Fy);
        const R F_w = R(2) * (ux * Fx - uy * Fy);
        const R F_xy = ux * Fy + uy * Fx;
        R Dm[9];
        Dm[0] = R(0);
        Dm[1] = R(3) * Fx;
        Dm[2] = R(3) * Fy;
        Dm[3] = P.frc[0] * F_e + P.rel[0] * (m[3] - eq_e);
        Dm[4] = P.frc[1] * F_w + P.rel[1] * (m[4] - eq_w);
        Dm[5] = P.frc[2] * F_xy + P.rel[2] * (m[5] - eq_xy);
        Dm[6] = P.rel[3] * m[6];
        Dm[7] = P.rel[4] * m[7];
        Dm[8] = P.rel[5] * m[8];
        if (P.noise) {
            const R sr = P.noise_local ? sqrt_(rho) : R(P.sqrt_rho0);
            R z[8];
            noise_normals<2>(P.key, site, step, P.replica, z);
#pragma unroll
            for (int k = 0; k < 6; ++k) Dm[3 + k] += P.ns[k] * (sr * z[k]);
        }
        add_back(Dm, g);
    }

    // Modified-equilibrium model (Sec. IV.C): no force; the equilibrium adds
    // pex = p - rho cs^2 to e (x 6) and eps (x -6) (Eq. (meq-yeo)) and the
    // square-gradient stress kappa (d_a rho d_b rho - |grad rho|^2 delta/2) to
    // p_ww and p_xy; e and eps take the coloured noise (xe, xp) given per site,
    // the other non-conserved modes their white noise.
    template <class R, class PR>
    __device__ __forceinline__ static void collide_swift(R g[9], R pex, R gx, R gy, R kappa, R xe, R xp,
                                                         const Coll<PR>& P, uint32_t site, uint32_t step)
    {
        R m[9];
        moments(g, m);
        const R rho = P.rho0 + m[0];
        const R ir = rcp_(rho);
        const R ux = m[1] * ir, uy = m[2] * ir;
        const R uxx = ux * ux, uyy = uy * uy;
        const R eq_e = R(3) * rho * (uxx + uyy) + R(6) * pex;
        const R eq_w = rho * (uxx - uyy) + kappa * (gx * gx - gy * gy);
        const R eq_xy = rho * ux * uy + kappa * gx * gy;
        const R eq_eps = R(-6) * pex;
        R Dm[9];
        Dm[0] = Dm[1] = Dm[2] = R(0);
        Dm[3] = P.rel[0] * (m[3] - eq_e);
        Dm[4] = P.rel[1] * (m[4] - eq_w);
        Dm[5] = P.rel[2] * (m[5] - eq_xy);
        Dm[6] = P.rel[3] * m[6];
        Dm[7] = P.rel[4] * m[7];
        Dm[8] = P.rel[5] * (m[8] - eq_eps);
        if (P.noise) {
            const R sr = P.noise_local ? sqrt_(rho) : R(P.sqrt_rho0);
            R z[8];
            noise_normals<2>(P.key, site, step, P.replica, z);
#pragma unroll
            for (int k = 1; k < 5; ++k) Dm[3 + k] += P.ns[k] * (sr * z[k]);
            // the coloured noise is built around rho0: sqrt(rho / rho0) for the local density
            const R sc = sr * rcp_(R(P.sqrt_rho0));
            Dm[3] += (sc * xe) * R(1.0 / 4.0);   // / N_e
            Dm[8] += (sc * xp) * R(1.0 / 16.0);  // / N_eps
        }
        add_back(Dm, g);
    }
};

// ---------------------------------------------------------------------------
// D3Q19.  Velocity order: 0 rest; 1,2 = +-x; 3,4 = +-y; 5,6 = +-z;
// 7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0) 11 (1,0,1) 12 (-1,0,-1)
// 13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1).
// Pair p = 1..9 joins velocities 2p-1 and 2p (c and -c).
// Modes (weighted Gram-Schmidt basis) and norms N_a:
//  0 1 (1); 1-3 cx, cy, cz (1/3); 4 c^2-1 (2/3); 5 3cx^2-c^2 (4/3);
//  6 cy^2-cz^2 (4/9); 7-9 cxcy, cycz, czcx (1/9); 10-12 (c^2-5/3)c_a (2/27);
//  13 (cy^2-cz^2)cx, 14 (cz^2-cx^2)cy, 15 (cx^2-cy^2)cz (2/9);
//  16 c^4-2c^2+1/3 (2/9); 17 (c^2-3/2)(3cx^2-c^2) (1/3); 18 (c^2-3/2)(cy^2-cz^2) (1/9).
// Weights 1/3, 1/18 (axis), 1/36 (edge).
// ---------------------------------------------------------------------------
struct D3Q19 {
    static constexpr int Q = 19, D = 3, NNC = 15, NCALL = 4, NCALL_ALL = 5;

    template <class R>
    __device__ __forceinline__ static void moments(const R g[19], R m[19])
    {
        const R s1 = g[1] + g[2], d1 = g[1] - g[2];
        const R s2 = g[3] + g[4], d2 = g[3] - g[4];
        const R s3 = g[5] + g[6], d3 = g[5] - g[6];
        const R s4 = g[7] + g[8], d4 = g[7] - g[8];
        const R s5 = g[9] + g[10], d5 = g[9] - g[10];
        const R s6 = g[11] + g[12], d6 = g[11] - g[12];
        const R s7 = g[13] + g[14], d7 = g[13] - g[14];
        const R s8 = g[15] + g[16], d8 = g[15] - g[16];
        const R s9 = g[17] + g[18], d9 = g[17] - g[18];
        const R sa = s1 + s2 + s3;               // axis pairs
        const R sxy = s4 + s5, sxz = s6 + s7, syz = s8 + s9;
        const R se = sxy + sxz + syz;            // edge pairs
        m[0] = g[0] + sa + se;
        m[1] = d1 + d4 + d5 + d6 + d7;
        m[2] = d2 + d4 - d5 + d8 + d9;
        m[3] = d3 + d6 - d7 + d8 - d9;
        m[4] = se - g[0];
        m[5] = R(2) * s1 - s2 - s3 + sxy + sxz - R(2) * syz;
        m[6] = s2 - s3 + sxy - sxz;
        m[7] = s4 - s5;
        m[8] = s8 - s9;
        m[9] = s6 - s7;
        m[10] = R(1.0 / 3.0) * (d4 + d5 + d6 + d7 - R(2) * d1);
        m[11] = R(1.0 / 3.0) * (d4 - d5 + d8 + d9 - R(2) * d2);
        m[12] = R(1.0 / 3.0) * (d6 - d7 + d8 - d9 - R(2) * d3);
        m[13] = d4 + d5 - d6 - d7;
        m[14] = d5 - d4 + d8 + d9;
        m[15] = d6 - d7 - d8 + d9;
        m[16] = R(1.0 / 3.0) * (g[0] + se - R(2) * sa);
        m[17] = R(0.5) * (s2 + s3 + sxy + sxz) - s1 - syz;
        m[18] = R(0.5) * (s3 - s2 + sxy - sxz);
    }

    // g_i += w_i sum_a T_ai D_a over the modes a >= 1 (J = false: the momentum
    // increments D_1..3 are zero and skipped).
    template <bool J = true, class R>
    __device__ __forceinline__ static void add_back(const R Dm[19], R g[19])
    {
        const R De = Dm[4], D5 = Dm[5], D6 = Dm[6], D7 = Dm[7], D8 = Dm[8], D9 = Dm[9];
        const R D10 = Dm[10], D11 = Dm[11], D12 = Dm[12], D13 = Dm[13], D14 = Dm[14], D15 = Dm[15];
        const R D16 = Dm[16], D17 = Dm[17], D18 = Dm[18];
        const R Jx = Dm[1], Jy = Dm[2], Jz = Dm[3];
        // odd parts without the momentum increments
        auto odd = [&](R j, R rest) { if constexpr (J) return j + rest; else return rest; };
        const R t16 = R(1.0 / 3.0) * D16, h17 = R(0.5) * D17, h18 = R(0.5) * D18;
        const R a10 = R(1.0 / 3.0) * D10, a11 = R(1.0 / 3.0) * D11, a12 = R(1.0 / 3.0) * D12;
        // rest particle: e = -1, c^4-2c^2+1/3 = 1/3
        g[0] += R(1.0 / 3.0) * (t16 - De);
        // axis pairs: e = 0, c^4-term = -2/3
        const R Ea = R(-2) * t16;
        const R E1 = Ea + R(2) * D5 - D17, O1 = odd(Jx, R(-2) * a10);
        const R E2 = Ea - D5 + D6 + h17 - h18, O2 = odd(Jy, R(-2) * a11);
        const R E3 = Ea - D5 - D6 + h17 + h18, O3 = odd(Jz, R(-2) * a12);
        // edge pairs: e = 1, c^4-term = 1/3
        const R Ee = De + t16;
        const R Exy = Ee + D5 + D6 + h17 + h18;
        const R E4 = Exy + D7, O4 = odd(Jx + Jy, a10 + a11 + D13 - D14);
        const R E5 = Exy - D7, O5 = odd(Jx - Jy, a10 - a11 + D13 + D14);
        const R Exz = Ee + D5 - D6 + h17 - h18;
        const R E6 = Exz + D9, O6 = odd(Jx + Jz, a10 + a12 - D13 + D15);
        const R E7 = Exz - D9, O7 = odd(Jx - Jz, a10 - a12 - D13 - D15);
        const R Eyz = Ee - R(2) * D5 - D17;
        const R E8 = Eyz + D8, O8 = odd(Jy + Jz, a11 + a12 + D14 - D15);
        const R E9 = Eyz - D8, O9 = odd(Jy - Jz, a11 - a12 + D14 + D15);
        constexpr double wa = 1.0 / 18.0, we = 1.0 / 36.0;
        g[1] += R(wa) * (E1 + O1);
        g[2] += R(wa) * (E1 - O1);
        g[3] += R(wa) * (E2 + O2);
        g[4] += R(wa) * (E2 - O2);
        g[5] += R(wa) * (E3 + O3);
        g[6] += R(wa) * (E3 - O3);
        g[7] += R(we) * (E4 + O4);
        g[8] += R(we) * (E4 - O4);
        g[9] += R(we) * (E5 + O5);
        g[10] += R(we) * (E5 - O5);
        g[11] += R(we) * (E6 + O6);
        g[12] += R(we) * (E6 - O6);
        g[13] += R(we) * (E7 + O7);
        g[14] += R(we) * (E7 - O7);
        g[15] += R(we) * (E8 + O8);
        g[16] += R(we) * (E8 - O8);
        g[17] += R(we) * (E9 + O9);
        g[18] += R(we) * (E9 - O9);
    }

    template <class R>
    __device__ __forceinline__ static void from_moments(const R Dm[19], R g[19])
    {
        for (int i = 0; i < 19; ++i) g[i] = R(0);
        add_back(Dm, g);
        g[0] += R(1.0 / 3.0) * Dm[0];
        for (int i = 1; i < 7; ++i) g[i] += R(1.0 / 18.0) * Dm[0];
        for (int i = 7; i < 19; ++i) g[i] += R(1.0 / 36.0) * Dm[0];
    }

    __host__ __device__ static constexpr double N(int a)
    {
        return a == 0 ? 1.0 : a < 4 ? 1.0 / 3 : a == 4 ? 2.0 / 3 : a == 5 ? 4.0 / 3 : a == 6 ? 4.0 / 9
             : a < 10 ? 1.0 / 9 : a < 13 ? 2.0 / 27 : a < 17 ? 2.0 / 9 : a == 17 ? 1.0 / 3 : 1.0 / 9;
    }

    // Moments of f^eq(rho, u) - w rho0 (Eq. (feq)); ghosts vanish.
    template <class R>
    __device__ __forceinline__ static void eq_moments(R drho, R rho, R ux, R uy, R uz, R m[19])
    {
        const R uu = ux * ux + uy * uy + uz * uz;
        m[0] = drho;
        m[1] = rho * ux;
        m[2] = rho * uy;
        m[3] = rho * uz;
        m[4] = rho * uu;
        m[5] = rho * (R(3) * ux * ux - uu);
        m[6] = rho * (uy * uy - uz * uz);
        m[7] = rho * ux * uy;
        m[8] = rho * uy * uz;
        m[9] = rho * uz * ux;
        for (int a = 10; a < 19; ++a) m[a] = R(0);
    }

    // FORCE = false: F = 0 (ideal gas); the force terms are not evaluated.
    // first (optional): receives the pre-collision mass deviation and
    // momentum m[0..3] = sum_i g_i, sum_i c_i g_i the collision forms anyway.
    // INTERLEAVED: the two-site noise draws its Philox calls round-major.
    template <bool FORCE = true, bool INTERLEAVED = false, class R, class PR>
    __device__ __forceinline__ static void collide(R g[19], R Fx, R Fy, R Fz, const Coll<PR>& P, uint32_t site,
                                                   uint32_t step, R* first = nullptr)
    {
        R m[19];
        moments(g, m);
        if (first) {
            first[0] = m[0];
            first[1] = m[1];
            first[2] = m[2];
            first[3] = m[3];
        }
        const R rho = P.rho0 + m[0];
        const R ir = rcp_(rho);
        R ux, uy, uz;
        if constexpr (FORCE) {
            ux = (m[1] + R(0.5) * Fx) * ir;
            uy = (m[2] + R(0.5) * Fy) * ir;
            uz = (m[3] + R(0.5) * Fz) * ir;
        } else {
            ux = m[1] * ir;
            uy = m[2] * ir;
            uz = m[3] * ir;
        }
        const R uxx = ux * ux, uyy = uy * uy, uzz = uz * uz, uu = uxx + uyy + uzz;
        R Dm[19];
        Dm[0] = R(0);
        // bulk: m^eq = rho u^2, m^F = 2 u.F
        // shear: m^eq = rho(3ux^2-u^2), rho(uy^2-uz^2), rho ux uy, rho uy uz, rho uz ux
        Dm[4] = P.rel[0] * (m[4] - rho * uu);
        Dm[5] = P.rel[1] * (m[5] - rho * (R(3) * uxx - uu));
        Dm[6] = P.rel[2] * (m[6] - rho * (uyy - uzz));
        Dm[7] = P.rel[3] * (m[7] - rho * (ux * uy));
        Dm[8] = P.rel[4] * (m[8] - rho * (uy * uz));
        Dm[9] = P.rel[5] * (m[9] - rho * (uz * ux));
        if constexpr (FORCE) {
            const R uFx = ux * Fx, uFy = uy * Fy, uFz = uz * Fz, uF = uFx + uFy + uFz;
            Dm[1] = R(3) * Fx;
            Dm[2] = R(3) * Fy;
            Dm[3] = R(3) * Fz;
            Dm[4] += P.frc[0] * (R(2) * uF);
            Dm[5] += P.frc[1] * (R(2) * (R(3) * uFx - uF));
            Dm[6] += P.frc[2] * (R(2) * (uFy - uFz));
            Dm[7] += P.frc[3] * (ux * Fy + uy * Fx);
            Dm[8] += P.frc[4] * (uy * Fz + uz * Fy);
            Dm[9] += P.frc[5] * (uz * Fx + ux * Fz);
        } else {
            Dm[1] = Dm[2] = Dm[3] = R(0);
        }
        // ghosts relax to 0
#pragma unroll
        for (int a = 10; a < 19; ++a) Dm[a] = P.rel[a - 4] * m[a];
        if (P.noise) {
            const R sr = P.noise_local ? sqrt_(rho) : R(P.sqrt_rho0);
            R z[16];
            if constexpr (std::is_same<R, F2>::value)
                noise_normals<4, INTERLEAVED>(P.key, site, step, P.replica, z);
            else
                noise_normals<4>(P.key, site, step, P.replica, z);
#pragma unroll
            for (int k = 0; k < 15; ++k) Dm[4 + k] += P.ns[k] * (sr * z[k]);
        }
        add_back<FORCE>(Dm, g);
    }
};

// ---------------------------------------------------------------------------
// Geometry helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap_once(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
__device__ __forceinline__ int wrap_any(int a, int n)
{
    while (a < 0) a += n;
    while (a >= n) a -= n;
    return a;
}

}  // namespace flb
