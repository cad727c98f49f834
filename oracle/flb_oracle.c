/*
 * flb_oracle.c -- plain FP64 CPU reference ("oracle") of the fluctuating
 * lattice Boltzmann (FLB) update of M. Gross, M. E. Cates, F. Varnik and
 * R. Adhikari, "Langevin theory of fluctuations in the discrete Boltzmann
 * equation" (arXiv 1012.3632).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load this file:
 * only tests/, __graft_entry__.smoke() and the cpu_baseline / reference leg of
 * bench.py call it.  It shares no code, header, table or constant generator
 * with the CUDA library under paper_1012_3632_gb300/csrc.
 *
 * Written for readability, not speed: every step is the paper's formula,
 * evaluated site by site in double precision, in the paper's order.
 *
 *   lattice + basis   Sec. III, Eqs. (moments), (moments-inv), (T-orthog);
 *                     D2Q9 table of App. B, Eq. (TD2Q9); D3Q19 by Gram-Schmidt
 *   equilibrium       Eq. (feq)
 *   forcing           Eq. (forcing-term), read as the Guo form (see below)
 *   update            Eq. (lbe-mom), with lambda^LB = omega (Sec. V)
 *   noise variance    Eq. (noise-lbe), Delta V = 1
 *   observables       Eq. (lbe-moments): rho = sum f, rho u = sum f c + F/2
 *   force model       App. A, Eq. (he-force) written as F = -rho grad mu
 *   structure factor  G_11(k) = <|delta rho(k)|^2>/V (Sec. IV, Eq. (g-correl))
 *
 * Readings of the paper taken here (the paper is silent or its print is
 * ambiguous):
 *   - Forcing: Phi_i = w_i [F.c_i/s2 + (uF+Fu):Q_i/(2 s2^2)] (force density F,
 *     no rho prefactor, s2^2 in the second term), which gives the moments
 *     {0, F, uF+Fu, 0...} used by Eqs. (force-mom) and (lbe-moments).
 *   - Noise prefactor (1 - lambda/2) (Eqs. (lbe-mom), (noise-lbe)); the
 *     variance added to mode a per step is rho kT (2-w_a) w_a N_a / s2.
 *   - rho in the noise amplitude is the local pre-collision density (Sec. VI
 *     asks for local values in inhomogeneous states); noise_rho_local = 0
 *     selects the reference density rho0 instead.
 *   - Derivative stencils (not fixed by the paper): isotropic lattice stencils
 *     grad phi = (1/s2) sum_i w_i c_i phi(x+c_i),
 *     lap  phi = (2/s2) sum_i w_i (phi(x+c_i) - phi(x)).
 *   - D3Q19 basis: Gram-Schmidt, under (p,q) = sum_i w_i p_i q_i, of
 *     1; cx,cy,cz; c^2; 3cx^2-c^2, cy^2-cz^2; cxcy, cycz, czcx; c^2 c_a (x3);
 *     (cy^2-cz^2)cx, (cz^2-cx^2)cy, (cx^2-cy^2)cz; c^4; c^2(3cx^2-c^2),
 *     c^2(cy^2-cz^2).
 *   - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 *     key = (seed lo, seed hi), counter = (site, step, call | tag<<8, replica),
 *     uniforms (x + 1/2) 2^-32, Box-Muller on words (0,1) and (2,3).
 *     Non-conserved mode k (0-based among non-conserved modes) takes normal
 *     k%4 of call k/4.  Tag 0: collision noise; tag 1: thermal initial state.
 *
 * Array layout: populations f[i*V + s], s = x + wx*(y + wy*z) (structure of
 * arrays, x fastest).  Arrays hold the paper's pre-collision f^LB(r,t).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_QMAX 19
#define ORC_PI 3.14159265358979323846

/* c_s,LB^2 of both D2Q9 and D3Q19, Sec. III. */
static const double S2 = 1.0 / 3.0;

enum { CLS_CONSERVED = 0, CLS_BULK = 1, CLS_SHEAR = 2, CLS_GHOST = 3 };

typedef struct {
    int Q, D;
    int c[ORC_QMAX][3];
    double w[ORC_QMAX];
    double T[ORC_QMAX][ORC_QMAX]; /* T[a][i] */
    double N[ORC_QMAX];
    int cls[ORC_QMAX];
} orc_lattice;

typedef struct {
    int Q;
    int X, Y, Z;                 /* global periodic lattice */
    int ox, oy, oz;              /* window origin (global coordinates) */
    int wx, wy, wz;              /* window extent; == X,Y,Z for the full lattice */
    double omega_shear, omega_bulk, omega_ghost;
    double kT, rho0;
    int noise_rho_local;
    int nonideal;
    double A, B, rho_c, kappa;   /* psi(rho) = A (rho-rho_c)^2/2 + B (rho-rho_c)^4/4 */
    int total;                   /* psi is the total bulk free energy f0 of App. A */
    int model;                   /* 0: force-based (App. A); 1: modified equilibrium (Sec. IV.C, D2Q9) */
    uint64_t seed;
    uint32_t replica;
} orc_params;

/* ------------------------------------------------------------------ */
/* Lattices and moment bases                                           */
/* ------------------------------------------------------------------ */

/* D2Q9, App. B: velocity order fixed by rows 2-3 of Eq. (TD2Q9). */
static void d2q9(orc_lattice* L)
{
    static const int c[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                                {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    /* Eq. (TD2Q9), typed row by row from the paper. */
    static const double T[9][9] = {
        {1, 1, 1, 1, 1, 1, 1, 1, 1},
        {0, 1, 0, -1, 0, 1, -1, -1, 1},
        {0, 0, 1, 0, -1, 1, 1, -1, -1},
        {-2, 1, 1, 1, 1, 4, 4, 4, 4},
        {0, 1, -1, 1, -1, 0, 0, 0, 0},
        {0, 0, 0, 0, 0, 1, -1, 1, -1},
        {0, -1, 0, 1, 0, 2, -2, -2, 2},
        {0, 0, -1, 0, 1, 2, 2, -2, -2},
        {2, -4, -4, -4, -4, 8, 8, 8, 8}};
    /* N_a column of Table I (App. B). */
    static const double N[9] = {1.0, 1.0 / 3, 1.0 / 3, 4.0, 4.0 / 9, 1.0 / 9, 2.0 / 3, 2.0 / 3, 16.0};
    static const int cls[9] = {CLS_CONSERVED, CLS_CONSERVED, CLS_CONSERVED, CLS_BULK, CLS_SHEAR,
                               CLS_SHEAR, CLS_GHOST, CLS_GHOST, CLS_GHOST};
    L->Q = 9;
    L->D = 2;
    for (int i = 0; i < 9; i++) {
        L->c[i][0] = c[i][0];
        L->c[i][1] = c[i][1];
        L->c[i][2] = 0;
        int c2 = c[i][0] * c[i][0] + c[i][1] * c[i][1];
        L->w[i] = (c2 == 0) ? 4.0 / 9 : (c2 == 1 ? 1.0 / 9 : 1.0 / 36);
    }
    for (int a = 0; a < 9; a++) {
        L->N[a] = N[a];
        L->cls[a] = cls[a];
        for (int i = 0; i < 9; i++) L->T[a][i] = T[a][i];
    }
}

/* D3Q19 polynomial list (before orthogonalisation), evaluated at velocity c. */
static double d3q19_poly(int a, const int* c)
{
    double x = c[0], y = c[1], z = c[2];
    double c2 = x * x + y * y + z * z;
    switch (a) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return c2;
    case 5: return 3 * x * x - c2;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return y * z;
    case 9: return z * x;
    case 10: return c2 * x;
    case 11: return c2 * y;
    case 12: return c2 * z;
    case 13: return (y * y - z * z) * x;
    case 14: return (z * z - x * x) * y;
    case 15: return (x * x - y * y) * z;
    case 16: return c2 * c2;
    case 17: return c2 * (3 * x * x - c2);
    default: return c2 * (y * y - z * z);
    }
}

/* D3Q19: rest, 6 axis and 12 edge velocities, weights 1/3, 1/18, 1/36; basis by
 * Gram-Schmidt under the weighted inner product of Eq. (T-orthog). */
static void d3q19(orc_lattice* L)
{
    static const int c[19][3] = {
        {0, 0, 0},
        {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
        {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    L->Q = 19;
    L->D = 3;
    for (int i = 0; i < 19; i++) {
        int c2 = 0;
        for (int d = 0; d < 3; d++) {
            L->c[i][d] = c[i][d];
            c2 += c[i][d] * c[i][d];
        }
        L->w[i] = (c2 == 0) ? 1.0 / 3 : (c2 == 1 ? 1.0 / 18 : 1.0 / 36);
    }
    for (int a = 0; a < 19; a++) {
        for (int i = 0; i < 19; i++) L->T[a][i] = d3q19_poly(a, L->c[i]);
        for (int b = 0; b < a; b++) {
            double dot = 0;
            for (int i = 0; i < 19; i++) dot += L->w[i] * L->T[a][i] * L->T[b][i];
            for (int i = 0; i < 19; i++) L->T[a][i] -= dot / L->N[b] * L->T[b][i];
        }
        double n = 0;
        for (int i = 0; i < 19; i++) n += L->w[i] * L->T[a][i] * L->T[a][i];
        L->N[a] = n;
        L->cls[a] = (a < 4) ? CLS_CONSERVED : (a == 4 ? CLS_BULK : (a < 10 ? CLS_SHEAR : CLS_GHOST));
    }
}

static int lattice_of(int Q, orc_lattice* L)
{
    if (Q == 9) {
        d2q9(L);
        return 0;
    }
    if (Q == 19) {
        d3q19(L);
        return 0;
    }
    return -1;
}

/* Export the lattice tables: c[Q*3], w[Q], T[Q*Q] (row a, column i), N[Q], cls[Q]. */
int orc_get_lattice(int Q, int* c, double* w, double* T, double* N, int* cls)
{
    orc_lattice L;
    if (lattice_of(Q, &L)) return -1;
    for (int i = 0; i < Q; i++) {
        for (int d = 0; d < 3; d++) c[3 * i + d] = L.c[i][d];
        w[i] = L.w[i];
    }
    for (int a = 0; a < Q; a++) {
        N[a] = L.N[a];
        cls[a] = L.cls[a];
        for (int i = 0; i < Q; i++) T[a * Q + i] = L.T[a][i];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Random numbers: Philox4x32-10 and Box-Muller                        */
/* ------------------------------------------------------------------ */

/* Philox4x32 with 10 rounds, as published by Salmon et al. (SC'11): each round
 * multiplies words 0 and 2 by the two round constants, and the high halves are
 * mixed with the other two words and the key; the key is bumped by the Weyl
 * constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)M0 * x0;
        uint64_t p1 = (uint64_t)M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        x0 = hi1 ^ x1 ^ k0;
        x1 = lo1;
        x2 = hi0 ^ x3 ^ k1;
        x3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

/* Four standard normals from one Philox call with counter
 * (site, step, call | tag<<8, replica) and key (seed lo, seed hi). */
void orc_normals4(uint64_t seed, uint32_t site, uint32_t step, uint32_t call, uint32_t tag,
                  uint32_t replica, double z[4])
{
    uint32_t ctr[4] = {site, step, call | (tag << 8), replica};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    double u[4];
    for (int k = 0; k < 4; k++) u[k] = ((double)r[k] + 0.5) * (1.0 / 4294967296.0);
    double rad0 = sqrt(-2.0 * log(u[0]));
    double rad1 = sqrt(-2.0 * log(u[2]));
    z[0] = rad0 * cos(2.0 * ORC_PI * u[1]);
    z[1] = rad0 * sin(2.0 * ORC_PI * u[1]);
    z[2] = rad1 * cos(2.0 * ORC_PI * u[3]);
    z[3] = rad1 * sin(2.0 * ORC_PI * u[3]);
}

/* The first n normals of the stream for (site, step, tag): normal k comes from
 * call k/4, position k%4. */
static void normals(const orc_params* p, uint32_t site, uint64_t step, uint32_t tag, int n, double* z)
{
    for (int b = 0; 4 * b < n; b++) {
        double zb[4];
        orc_normals4(p->seed, site, (uint32_t)step, (uint32_t)b, tag, p->replica, zb);
        for (int r = 0; r < 4 && 4 * b + r < n; r++) z[4 * b + r] = zb[r];
    }
}

/* ------------------------------------------------------------------ */
/* Geometry                                                            */
/* ------------------------------------------------------------------ */

static long nsites(const orc_params* p) { return (long)p->wx * p->wy * p->wz; }

static int posmod(int a, int n) { return ((a % n) + n) % n; }

/* Window index of the site at local (x,y,z) + d, or -1 when it lies outside the
 * window.  Axes that the window covers entirely are periodic. */
static long nbr(const orc_params* p, int x, int y, int z, int dx, int dy, int dz)
{
    int l[3] = {x + dx, y + dy, z + dz};
    int w[3] = {p->wx, p->wy, p->wz};
    int G[3] = {p->X, p->Y, p->Z};
    for (int d = 0; d < 3; d++) {
        if (w[d] == G[d])
            l[d] = posmod(l[d], G[d]);
        else if (l[d] < 0 || l[d] >= w[d])
            return -1;
    }
    return l[0] + (long)p->wx * (l[1] + (long)p->wy * l[2]);
}

/* Global site index of local (x,y,z): keys the noise. */
static uint32_t global_site(const orc_params* p, int x, int y, int z)
{
    long gx = posmod(p->ox + x, p->X), gy = posmod(p->oy + y, p->Y), gz = posmod(p->oz + z, p->Z);
    return (uint32_t)(gx + (long)p->X * (gy + (long)p->Y * gz));
}

static int check_params(const orc_params* p, orc_lattice* L)
{
    if (lattice_of(p->Q, L)) return -1;
    if (p->X < 1 || p->Y < 1 || p->Z < 1 || p->wx < 1 || p->wy < 1 || p->wz < 1) return -1;
    if (p->wx > p->X || p->wy > p->Y || p->wz > p->Z) return -1;
    if (p->Q == 9 && p->Z != 1) return -1;
    if (p->nonideal && p->model == 1 &&
        (p->Q != 9 || p->wx != p->X || p->wy != p->Y || p->wz != p->Z))
        return -1; /* modified equilibrium: D2Q9, full lattice (its noise lives in k-space) */
    return 0;
}

/* ------------------------------------------------------------------ */
/* Equilibrium, forcing, collision                                     */
/* ------------------------------------------------------------------ */

static double relax_rate(const orc_params* p, int cls)
{
    switch (cls) {
    case CLS_BULK: return p->omega_bulk;
    case CLS_SHEAR: return p->omega_shear;
    case CLS_GHOST: return p->omega_ghost;
    default: return 0.0; /* conserved modes, Eq. (relax-eigenv) */
    }
}

/* Eq. (feq): second-order discrete Maxwellian. */
static void feq(const orc_lattice* L, double rho, const double u[3], double out[])
{
    double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < L->Q; i++) {
        double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
        double uuQ = cu * cu - S2 * u2; /* u_a u_b Q_iab */
        out[i] = L->w[i] * (rho + rho * cu / S2 + rho * uuQ / (2 * S2 * S2));
    }
}

/* Eq. (forcing-term) in the Guo reading stated in the header. */
static void forcing(const orc_lattice* L, const double u[3], const double F[3], double out[])
{
    double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    for (int i = 0; i < L->Q; i++) {
        double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
        double cF = L->c[i][0] * F[0] + L->c[i][1] * F[1] + L->c[i][2] * F[2];
        double uFQ = 2 * cu * cF - 2 * S2 * uF; /* (u_a F_b + F_a u_b) Q_iab */
        out[i] = L->w[i] * (cF / S2 + uFQ / (2 * S2 * S2));
    }
}

/* One site of Eq. (lbe-mom): f (pre-collision f^LB) -> fstar (post-collision),
 * before streaming.  F is the body force at the site; site/step key the noise. */
/* sw (modified-equilibrium model only, else NULL): {p - rho s2, d_x rho,
 * d_y rho, xi_e, xi_eps} at the site; see swift_fields(). */
static void collide(const orc_params* p, const orc_lattice* L, const double f[], const double F[3],
                    uint32_t site, uint64_t step, const double* sw, double fstar[])
{
    int Q = L->Q;
    double m[ORC_QMAX], meq[ORC_QMAX], mF[ORC_QMAX], ms[ORC_QMAX];
    double fe[ORC_QMAX], phi[ORC_QMAX];

    /* Eq. (moments) */
    for (int a = 0; a < Q; a++) {
        m[a] = 0;
        for (int i = 0; i < Q; i++) m[a] += L->T[a][i] * f[i];
    }
    /* Eq. (lbe-moments): rho = sum f, rho u = sum f c + F/2 */
    double rho = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; i++) {
        rho += f[i];
        for (int d = 0; d < 3; d++) j[d] += f[i] * L->c[i][d];
    }
    double u[3];
    for (int d = 0; d < 3; d++) u[d] = (j[d] + 0.5 * F[d]) / rho;

    feq(L, rho, u, fe);
    forcing(L, u, F, phi);
    for (int a = 0; a < Q; a++) {
        meq[a] = 0;
        mF[a] = 0;
        for (int i = 0; i < Q; i++) {
            meq[a] += L->T[a][i] * fe[i];
            mF[a] += L->T[a][i] * phi[i];
        }
    }
    if (sw) {
        /* Eq. (meq-yeo) with the pressure p = p0(rho) - kappa rho lap rho and the
         * square-gradient stress kappa (d_a rho d_b rho - |grad rho|^2 delta_ab / 2)
         * in the equilibrium: e gets 6 (p - rho s2), eps gets -6 (p - rho s2),
         * p_ww and p_xy the deviatoric stress.  D2Q9 mode order of App. B. */
        meq[3] += 6.0 * sw[0];
        meq[8] -= 6.0 * sw[0];
        meq[4] += p->kappa * (sw[1] * sw[1] - sw[2] * sw[2]);
        meq[5] += p->kappa * sw[1] * sw[2];
    }

    double rho_n = p->noise_rho_local ? rho : p->rho0;
    double z[ORC_QMAX];
    normals(p, site, step, 0, Q - 1 - L->D, z); /* one normal per non-conserved mode */
    int k = 0; /* index among non-conserved modes */
    for (int a = 0; a < Q; a++) {
        double om = relax_rate(p, L->cls[a]);
        double xi = 0.0;
        if (L->cls[a] != CLS_CONSERVED) {
            /* Eq. (noise-lbe): variance rho kT (2-omega) omega N_a / s2, Delta V = 1 */
            double var = rho_n * p->kT * (2.0 - om) * om * L->N[a] / S2;
            xi = sqrt(var) * z[k];
            /* modified equilibrium: e and eps carry the k-dependent noise, built
             * around rho0 and scaled by sqrt(rho / rho0) for the local density
             * (Sec. VI: local values in inhomogeneous states) */
            if (sw && (a == 3 || a == 8)) {
                double sc = p->noise_rho_local ? sqrt(rho / p->rho0) : 1.0;
                xi = sc * (a == 3 ? sw[3] : sw[4]);
            }
            k++;
        }
        ms[a] = m[a] - om * (m[a] - meq[a]) + (1.0 - 0.5 * om) * mF[a] + xi;
    }
    /* Eq. (moments-inv) */
    for (int i = 0; i < Q; i++) {
        fstar[i] = 0;
        for (int a = 0; a < Q; a++) fstar[i] += L->w[i] * L->T[a][i] * ms[a] / L->N[a];
    }
}

/* Single-site collision for unit tests: f, F in, fstar out. */
int orc_collide_site(const orc_params* p, const double* f, const double* F, uint32_t site,
                     uint64_t step, double* fstar)
{
    orc_lattice L;
    if (lattice_of(p->Q, &L)) return -1;
    double F3[3] = {F[0], F[1], L.D == 3 ? F[2] : 0.0};
    collide(p, &L, f, F3, site, step, NULL, fstar);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Non-ideal force: F = -rho grad mu, mu = psi'(rho) - kappa lap rho     */
/* ------------------------------------------------------------------ */

static double psi_prime(const orc_params* p, double rho)
{
    double d = rho - p->rho_c;
    return p->A * d + p->B * d * d * d;
}

/* rho[V], F[3V] of the state f.  Sites whose stencil leaves the window get NaN.
 * For the ideal gas F = 0.
 *
 * psi the excess free energy over the ideal lattice gas (default):
 *   F = -rho grad mu.
 * psi the total bulk free energy f0 (total = 1), Eq. (he-force) as printed:
 *   F = kappa rho grad lap rho - grad(p0 - rho s2) with grad p0 = rho grad f0'
 *     = -rho grad mu + s2 grad rho,
 * the last term cancelling the ideal-gas pressure the LB carries itself. */
static void density_force(const orc_params* p, const orc_lattice* L, const double* f, double* rho,
                          double* F)
{
    long V = nsites(p);
    for (long s = 0; s < V; s++) {
        rho[s] = 0;
        for (int i = 0; i < L->Q; i++) rho[s] += f[i * V + s];
        F[s] = F[V + s] = F[2 * V + s] = 0.0;
    }
    if (!p->nonideal || p->model == 1) return;

    double* mu = (double*)malloc(sizeof(double) * V);
    for (int z = 0; z < p->wz; z++)
        for (int y = 0; y < p->wy; y++)
            for (int x = 0; x < p->wx; x++) {
                long s = x + (long)p->wx * (y + (long)p->wy * z);
                double lap = 0;
                for (int i = 0; i < L->Q; i++) {
                    long n = nbr(p, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
                    lap += L->w[i] * ((n < 0 ? NAN : rho[n]) - rho[s]);
                }
                lap *= 2.0 / S2;
                mu[s] = psi_prime(p, rho[s]) - p->kappa * lap;
            }
    for (int z = 0; z < p->wz; z++)
        for (int y = 0; y < p->wy; y++)
            for (int x = 0; x < p->wx; x++) {
                long s = x + (long)p->wx * (y + (long)p->wy * z);
                double g[3] = {0, 0, 0};
                for (int i = 0; i < L->Q; i++) {
                    long n = nbr(p, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
                    double mun = (n < 0) ? NAN : mu[n];
                    for (int d = 0; d < 3; d++) g[d] += L->w[i] * L->c[i][d] * mun;
                }
                for (int d = 0; d < 3; d++) F[d * V + s] = -rho[s] * g[d] / S2;
                if (p->total) {
                    double gr[3] = {0, 0, 0};
                    for (int i = 0; i < L->Q; i++) {
                        long n = nbr(p, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
                        double rn = (n < 0) ? NAN : rho[n];
                        for (int d = 0; d < 3; d++) gr[d] += L->w[i] * L->c[i][d] * rn;
                    }
                    for (int d = 0; d < 3; d++) F[d * V + s] += S2 * (gr[d] / S2);
                }
            }
    free(mu);
}

int orc_density_force(const orc_params* p, const double* f, double* rho, double* F)
{
    orc_lattice L;
    if (check_params(p, &L)) return -1;
    density_force(p, &L, f, rho, F);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Time step, Eq. (lbe-gen) / (lbe-mom): collide at r, move to r + c_i  */
/* ------------------------------------------------------------------ */

int orc_dft(int nx, int ny, int nz, const double* phi, double* out_re, double* out_im);

/* ------------------------------------------------------------------ */
/* Modified-equilibrium model (Sec. IV.C), D2Q9                          */
/* ------------------------------------------------------------------ */

/* Bulk pressure minus the ideal lattice-gas pressure, p0(rho) - rho s2, with
 * p0 = rho psi' - psi (+ rho s2 when psi is the excess free energy). */
static double p0_excess(const orc_params* p, double rho)
{
    double d = rho - p->rho_c;
    double psi = 0.5 * p->A * d * d + 0.25 * p->B * d * d * d * d;
    double v = rho * psi_prime(p, rho) - psi;
    return p->total ? v - rho * S2 : v;
}

/* c_s^2 = d p0 / d rho at rho0 (the speed of sound of Eq. (s-nonideal)). */
static double cs2_rho0(const orc_params* p)
{
    double d = p->rho0 - p->rho_c;
    double psi2 = p->A + 3.0 * p->B * d * d;
    return p->rho0 * psi2 + (p->total ? 0.0 : S2);
}

/* In-place inverse DFT of a complex nx*ny field: phi(r) = (1/V) sum_k phi(k) e^{ik.r},
 * direct sums along x, then y. */
static void idft2(int nx, int ny, double* re, double* im)
{
    int n[2] = {nx, ny};
    long stride[2] = {1, nx};
    long V = (long)nx * ny;
    int Lmax = nx > ny ? nx : ny;
    double* lr = (double*)malloc(sizeof(double) * Lmax);
    double* li = (double*)malloc(sizeof(double) * Lmax);
    for (int ax = 0; ax < 2; ax++) {
        int L = n[ax];
        if (L == 1) continue;
        for (long base = 0; base < V; base++) {
            if ((base / stride[ax]) % L != 0) continue;
            for (int r = 0; r < L; r++) {
                double a = 0, b = 0;
                for (int k = 0; k < L; k++) {
                    double t = 2.0 * ORC_PI * (double)(((long)k * r) % L) / L;
                    double x = re[base + k * stride[ax]], y = im[base + k * stride[ax]];
                    a += x * cos(t) - y * sin(t); /* (x + iy)(cos + i sin) */
                    b += x * sin(t) + y * cos(t);
                }
                lr[r] = a;
                li[r] = b;
            }
            for (int r = 0; r < L; r++) {
                re[base + r * stride[ax]] = lr[r];
                im[base + r * stride[ax]] = li[r];
            }
        }
    }
    for (long s = 0; s < V; s++) {
        re[s] /= V;
        im[s] /= V;
    }
    free(lr);
    free(li);
}

/* Per-site inputs of the modified-equilibrium collision, sw[5 s + 0..4] =
 * {p - rho s2, d_x rho, d_y rho, xi_e, xi_eps}:
 *   p = p0(rho) - kappa rho lap rho (isotropic stencils);
 *   (xi_e, xi_eps): Gaussian field with, at each k = 2 pi n / L, the 2x2
 *   covariance of the e and eps modes of the lattice noise (Eq. (noise-yeo)
 *   under the map of Sec. V: xi^LB = (1 - omega/2) xi, lambda = 2 omega/(2 - omega)),
 *   c_s^2(k) = c_s^2 + kappa rho0 K2(k), K2(k) = (2/s2) sum_i w_i (1 - cos k.c_i),
 *   made from the white normals z_e, z_eps of the collision draw (modes e and
 *   eps, i.e. normals 0 and 5 of the site) by xi(k) = C(k) z(k), C C^T the
 *   covariance (lower Cholesky factor), and an inverse DFT.
 * Returns -1 where the covariance is not positive definite. */
static int swift_fields(const orc_params* p, const orc_lattice* L, const double* rho, uint64_t step, double* sw)
{
    int X = p->X, Y = p->Y;
    long V = (long)X * Y;
    for (int y = 0; y < Y; y++)
        for (int x = 0; x < X; x++) {
            long s = x + (long)X * y;
            double lap = 0, g[2] = {0, 0};
            for (int i = 0; i < L->Q; i++) {
                long n = nbr(p, x, y, 0, L->c[i][0], L->c[i][1], 0);
                lap += L->w[i] * (rho[n] - rho[s]);
                for (int d = 0; d < 2; d++) g[d] += L->w[i] * L->c[i][d] * rho[n];
            }
            lap *= 2.0 / S2;
            sw[5 * s + 0] = p0_excess(p, rho[s]) - p->kappa * rho[s] * lap;
            sw[5 * s + 1] = g[0] / S2;
            sw[5 * s + 2] = g[1] / S2;
            sw[5 * s + 3] = sw[5 * s + 4] = 0.0;
        }
    if (p->kT == 0.0) return 0;

    double* er = (double*)malloc(sizeof(double) * V);
    double* ei = (double*)malloc(sizeof(double) * V);
    double* pr = (double*)malloc(sizeof(double) * V);
    double* pi = (double*)malloc(sizeof(double) * V);
    double* ze = (double*)malloc(sizeof(double) * V);
    double* zp = (double*)malloc(sizeof(double) * V);
    for (int y = 0; y < Y; y++)
        for (int x = 0; x < X; x++) {
            double z[8];
            normals(p, global_site(p, x, y, 0), step, 0, L->Q - 1 - L->D, z);
            ze[x + (long)X * y] = z[0];
            zp[x + (long)X * y] = z[5];
        }
    orc_dft(X, Y, 1, ze, er, ei);
    orc_dft(X, Y, 1, zp, pr, pi);
    double oe = p->omega_bulk, op = p->omega_ghost;
    double le = 2.0 * oe / (2.0 - oe), lp = 2.0 * op / (2.0 - op);
    double se = 1.0 - 0.5 * oe, sp = 1.0 - 0.5 * op;
    double pre = 2.0 * p->rho0 * p->kT / S2, cs2 = cs2_rho0(p);
    int bad = 0;
    for (int ny = 0; ny < Y; ny++)
        for (int nx = 0; nx < X; nx++) {
            long s = nx + (long)X * ny;
            double kx = 2.0 * ORC_PI * nx / X, ky = 2.0 * ORC_PI * ny / Y, K2 = 0;
            for (int i = 0; i < L->Q; i++) K2 += L->w[i] * (1.0 - cos(kx * L->c[i][0] + ky * L->c[i][1]));
            K2 *= 2.0 / S2;
            double c2 = cs2 + p->kappa * p->rho0 * K2;
            double a = se * se * pre * L->N[3] * (2.0 - 3.0 * c2) * le;
            double c = sp * sp * pre * L->N[8] * (1.25 - 0.75 * c2) * lp;
            double b = se * sp * pre * 6.0 * (c2 - S2) * (le + lp);
            if (!(a > 0) || !(c - b * b / a >= 0)) bad = 1;
            double c11 = sqrt(a > 0 ? a : 0), c21 = a > 0 ? b / c11 : 0;
            double c22 = sqrt(c - c21 * c21 > 0 ? c - c21 * c21 : 0);
            double e_r = c11 * er[s], e_i = c11 * ei[s];
            double p_r = c21 * er[s] + c22 * pr[s], p_i = c21 * ei[s] + c22 * pi[s];
            er[s] = e_r;
            ei[s] = e_i;
            pr[s] = p_r;
            pi[s] = p_i;
        }
    idft2(X, Y, er, ei);
    idft2(X, Y, pr, pi);
    for (long s = 0; s < V; s++) {
        sw[5 * s + 3] = er[s];
        sw[5 * s + 4] = pr[s];
    }
    free(er);
    free(ei);
    free(pr);
    free(pi);
    free(ze);
    free(zp);
    return bad ? -1 : 0;
}

int orc_step(const orc_params* p, uint64_t step, const double* f, double* fnew)
{
    orc_lattice L;
    if (check_params(p, &L)) return -1;
    long V = nsites(p);
    int Q = L.Q;
    double* rho = (double*)malloc(sizeof(double) * V);
    double* F = (double*)malloc(sizeof(double) * 3 * V);
    density_force(p, &L, f, rho, F);
    for (long n = 0; n < (long)Q * V; n++) fnew[n] = NAN; /* sites fed from outside the window */
    double* sw = NULL;
    if (p->nonideal && p->model == 1) {
        sw = (double*)malloc(sizeof(double) * 5 * V);
        if (swift_fields(p, &L, rho, step, sw)) {
            free(sw);
            free(rho);
            free(F);
            return -1;
        }
    }

    for (int z = 0; z < p->wz; z++)
        for (int y = 0; y < p->wy; y++)
            for (int x = 0; x < p->wx; x++) {
                long s = x + (long)p->wx * (y + (long)p->wy * z);
                double fs[ORC_QMAX], fst[ORC_QMAX], Fs[3];
                for (int i = 0; i < Q; i++) fs[i] = f[i * V + s];
                for (int d = 0; d < 3; d++) Fs[d] = F[d * V + s];
                collide(p, &L, fs, Fs, global_site(p, x, y, z), step, sw ? sw + 5 * s : NULL, fst);
                for (int i = 0; i < Q; i++) {
                    long n = nbr(p, x, y, z, L.c[i][0], L.c[i][1], L.c[i][2]);
                    if (n >= 0) fnew[i * V + n] = fst[i];
                }
            }
    free(sw);
    free(rho);
    free(F);
    return 0;
}

/* nsteps updates starting at time step0; f is updated in place. */
int orc_run(const orc_params* p, uint64_t step0, int nsteps, double* f)
{
    orc_lattice L;
    if (check_params(p, &L)) return -1;
    long n = (long)L.Q * nsites(p);
    double* tmp = (double*)malloc(sizeof(double) * n);
    for (int t = 0; t < nsteps; t++) {
        int rc = orc_step(p, step0 + (uint64_t)t, f, tmp);
        if (rc) {
            free(tmp);
            return rc;
        }
        memcpy(f, tmp, sizeof(double) * n);
    }
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Initial state                                                       */
/* ------------------------------------------------------------------ */

/* f = f^eq(rho, u) (Eq. (feq)); with thermal != 0 every mode a additionally gets
 * a Gaussian of variance rho kT N_a / s2, the equal-time variance G_aa of
 * Eqs. (G-ideal), (mu-ideal), drawn with tag 1 at step 0. rho (V) and u (D*V)
 * may be NULL: rho0 and rest. */
int orc_init(const orc_params* p, const double* rho, const double* u, int thermal, double* f)
{
    orc_lattice L;
    if (check_params(p, &L)) return -1;
    long V = nsites(p);
    int Q = L.Q;
    for (int z = 0; z < p->wz; z++)
        for (int y = 0; y < p->wy; y++)
            for (int x = 0; x < p->wx; x++) {
                long s = x + (long)p->wx * (y + (long)p->wy * z);
                double r = rho ? rho[s] : p->rho0;
                double us[3] = {0, 0, 0};
                if (u)
                    for (int d = 0; d < L.D; d++) us[d] = u[d * V + s];
                double fe[ORC_QMAX], dm[ORC_QMAX];
                feq(&L, r, us, fe);
                double rn = p->noise_rho_local ? r : p->rho0;
                double zt[ORC_QMAX];
                normals(p, global_site(p, x, y, z), 0, 1, Q, zt); /* one normal per mode, tag 1 */
                for (int a = 0; a < Q; a++)
                    dm[a] = thermal ? sqrt(rn * p->kT * L.N[a] / S2) * zt[a] : 0.0;
                for (int i = 0; i < Q; i++) {
                    double df = 0;
                    for (int a = 0; a < Q; a++) df += L.w[i] * L.T[a][i] * dm[a] / L.N[a];
                    f[i * V + s] = fe[i] + df;
                }
            }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Observables                                                         */
/* ------------------------------------------------------------------ */

/* m[a*V + s] = sum_i T_ai f_i(s), Eq. (moments). */
int orc_modes(const orc_params* p, const double* f, double* m)
{
    orc_lattice L;
    if (check_params(p, &L)) return -1;
    long V = nsites(p);
    for (int a = 0; a < L.Q; a++)
        for (long s = 0; s < V; s++) {
            double acc = 0;
            for (int i = 0; i < L.Q; i++) acc += L.T[a][i] * f[i * V + s];
            m[a * V + s] = acc;
        }
    return 0;
}

/* Physical velocity u = (sum f c + F/2) / rho, Eq. (lbe-moments); u[d*V + s]. */
int orc_velocity(const orc_params* p, const double* f, double* u)
{
    orc_lattice L;
    if (check_params(p, &L)) return -1;
    long V = nsites(p);
    double* rho = (double*)malloc(sizeof(double) * V);
    double* F = (double*)malloc(sizeof(double) * 3 * V);
    density_force(p, &L, f, rho, F);
    for (long s = 0; s < V; s++)
        for (int d = 0; d < L.D; d++) {
            double j = 0;
            for (int i = 0; i < L.Q; i++) j += f[i * V + s] * L.c[i][d];
            u[d * V + s] = (j + 0.5 * F[d * V + s]) / rho[s];
        }
    free(rho);
    free(F);
    return 0;
}

/* Naive separable discrete Fourier transform of a real field phi on an
 * nx*ny*nz periodic grid: out(k) = sum_r phi(r) exp(-i k.r), k = 2 pi n / L.
 * Direct O(L^2) sums along x, then y, then z. */
int orc_dft(int nx, int ny, int nz, const double* phi, double* out_re, double* out_im)
{
    long V = (long)nx * ny * nz;
    for (long s = 0; s < V; s++) {
        out_re[s] = phi[s];
        out_im[s] = 0.0;
    }
    int n[3] = {nx, ny, nz};
    long stride[3] = {1, nx, (long)nx * ny};
    int Lmax = nx > ny ? nx : ny;
    if (nz > Lmax) Lmax = nz;
    double* lr = (double*)malloc(sizeof(double) * Lmax);
    double* li = (double*)malloc(sizeof(double) * Lmax);
    double* cs = (double*)malloc(sizeof(double) * Lmax);
    double* sn = (double*)malloc(sizeof(double) * Lmax);
    for (int ax = 0; ax < 3; ax++) {
        int L = n[ax];
        if (L == 1) continue;
        for (int m = 0; m < L; m++) {
            cs[m] = cos(2.0 * ORC_PI * m / L);
            sn[m] = sin(2.0 * ORC_PI * m / L);
        }
        for (long base = 0; base < V; base++) {
            /* visit each line once: its first element has coordinate 0 on ax */
            if ((base / stride[ax]) % L != 0) continue;
            for (int k = 0; k < L; k++) {
                double re = 0, im = 0;
                for (int r = 0; r < L; r++) {
                    int m = (int)(((long)k * r) % L);
                    double a = out_re[base + r * stride[ax]], b = out_im[base + r * stride[ax]];
                    /* (a + ib) (cos - i sin) */
                    re += a * cs[m] + b * sn[m];
                    im += b * cs[m] - a * sn[m];
                }
                lr[k] = re;
                li[k] = im;
            }
            for (int k = 0; k < L; k++) {
                out_re[base + k * stride[ax]] = lr[k];
                out_im[base + k * stride[ax]] = li[k];
            }
        }
    }
    free(lr);
    free(li);
    free(cs);
    free(sn);
    return 0;
}

/* S_a(k) = |sum_r dm_a(r) e^{-ik.r}|^2 / V with dm_a = m_a - mean_r(m_a);
 * mode 0 is the density, giving the structure factor G_11(k) of Eq. (g-correl).
 * Full lattice only. */
int orc_structure_factor(const orc_params* p, const double* f, int mode, double* S)
{
    orc_lattice L;
    if (check_params(p, &L)) return -1;
    if (p->wx != p->X || p->wy != p->Y || p->wz != p->Z) return -1;
    if (mode < 0 || mode >= L.Q) return -1;
    long V = nsites(p);
    double* m = (double*)malloc(sizeof(double) * V);
    double* re = (double*)malloc(sizeof(double) * V);
    double* im = (double*)malloc(sizeof(double) * V);
    double mean = 0;
    for (long s = 0; s < V; s++) {
        double acc = 0;
        for (int i = 0; i < L.Q; i++) acc += L.T[mode][i] * f[i * V + s];
        m[s] = acc;
        mean += acc;
    }
    mean /= (double)V;
    for (long s = 0; s < V; s++) m[s] -= mean;
    orc_dft(p->X, p->Y, p->Z, m, re, im);
    for (long s = 0; s < V; s++) S[s] = (re[s] * re[s] + im[s] * im[s]) / (double)V;
    free(m);
    free(re);
    free(im);
    return 0;
}
