/*
 * Seeded synthetic inputs for the domain-wall multigrid solver: a
 * counter-based random number generator, Gaussian fields and a quenched
 * Wilson-gauge heatbath for SU(3) links.
 *
 * This file holds no arithmetic of the solver itself.  It produces the
 * gauge fields and random vectors that both the GPU path and the FP64
 * oracle consume, so that the two see identical inputs.
 *
 * Lattice conventions shared with every consumer:
 *   4D site index  = ((t*Z + z)*Y + y)*X + x   (x fastest)
 *   links          = U[site][mu][a][b], mu = 0..3 for x,y,z,t, complex128,
 *                    row-major 3x3 (a = row, b = column)
 *   gauge boundary = periodic in all four directions
 *
 * Random numbers: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11).  Every draw is addressed by
 * (key = (seed, stream), counter = (c0, c1, c2, c3)), so results do not
 * depend on thread count or iteration order.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* ------------------------------------------------------------------ */
/* Philox-4x32-10                                                      */
/* ------------------------------------------------------------------ */

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static inline void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void dwfin_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k);
        k[0] += PHILOX_W0;
        k[1] += PHILOX_W1;
    }
    memcpy(out, c, sizeof(c));
}

/* Two uniform doubles in the open interval (0, 1), 53 bits each, from one
 * Philox block. */
static inline void uniform2(const uint32_t ctr[4], const uint32_t key[2], double u[2])
{
    uint32_t r[4];
    dwfin_philox4x32_10(ctr, key, r);
    const double inv53 = 1.0 / 9007199254740992.0;
    u[0] = ((double)(r[0] >> 5) * 67108864.0 + (double)(r[1] >> 6) + 0.5) * inv53;
    u[1] = ((double)(r[2] >> 5) * 67108864.0 + (double)(r[3] >> 6) + 0.5) * inv53;
}

/* Box-Muller: two independent N(0,1) numbers. */
static inline void gauss2(const uint32_t ctr[4], const uint32_t key[2], double g[2])
{
    double u[2];
    uniform2(ctr, key, u);
    double r = sqrt(-2.0 * log(u[0]));
    double th = 6.283185307179586476925286766559 * u[1];
    g[0] = r * cos(th);
    g[1] = r * sin(th);
}

/* n uniform doubles in (0,1): element i uses counter (i/2, c1, c2, c3). */
void dwfin_uniform(double *out, int64_t n, uint32_t seed, uint32_t stream, uint32_t c1,
                   uint32_t c2)
{
    const uint32_t key[2] = {seed, stream};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (n + 1) / 2; ++i) {
        uint32_t ctr[4] = {(uint32_t)i, c1, c2, (uint32_t)(i >> 32)};
        double u[2];
        uniform2(ctr, key, u);
        out[2 * i] = u[0];
        if (2 * i + 1 < n) out[2 * i + 1] = u[1];
    }
}

/* n complex numbers with real and imaginary parts i.i.d. N(0, sigma^2). */
void dwfin_gauss_complex(double *out, int64_t n, double sigma, uint32_t seed, uint32_t stream)
{
    const uint32_t key[2] = {seed, stream};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint32_t ctr[4] = {(uint32_t)i, 0u, 0u, (uint32_t)(i >> 32)};
        double g[2];
        gauss2(ctr, key, g);
        out[2 * i] = sigma * g[0];
        out[2 * i + 1] = sigma * g[1];
    }
}

/* ------------------------------------------------------------------ */
/* SU(3) helpers                                                       */
/* ------------------------------------------------------------------ */

/* Project a 3x3 matrix onto SU(3): normalise row 0, orthogonalise and
 * normalise row 1, set row 2 = conj(row0 x row1).  Leaves det = 1 and
 * makes row 2 exactly the one a two-row (12 real) storage rebuilds. */
void dwfin_project_su3(cplx m[9])
{
    cplx *r0 = m, *r1 = m + 3, *r2 = m + 6;
    double n0 = sqrt(creal(r0[0] * conj(r0[0]) + r0[1] * conj(r0[1]) + r0[2] * conj(r0[2])));
    for (int i = 0; i < 3; ++i) r0[i] /= n0;
    cplx d = conj(r0[0]) * r1[0] + conj(r0[1]) * r1[1] + conj(r0[2]) * r1[2];
    for (int i = 0; i < 3; ++i) r1[i] -= d * r0[i];
    double n1 = sqrt(creal(r1[0] * conj(r1[0]) + r1[1] * conj(r1[1]) + r1[2] * conj(r1[2])));
    for (int i = 0; i < 3; ++i) r1[i] /= n1;
    r2[0] = conj(r0[1] * r1[2] - r0[2] * r1[1]);
    r2[1] = conj(r0[2] * r1[0] - r0[0] * r1[2]);
    r2[2] = conj(r0[0] * r1[1] - r0[1] * r1[0]);
}

void dwfin_project_su3_field(double *U, int64_t nmat)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nmat; ++i) dwfin_project_su3((cplx *)U + 9 * i);
}

static inline void mul33(cplx c[9], const cplx a[9], const cplx b[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

/* c = a * b^dagger */
static inline void mul33_nd(cplx c[9], const cplx a[9], const cplx b[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            c[3 * i + j] = a[3 * i] * conj(b[3 * j]) + a[3 * i + 1] * conj(b[3 * j + 1]) +
                           a[3 * i + 2] * conj(b[3 * j + 2]);
}

/* c = a^dagger * b */
static inline void mul33_dn(cplx c[9], const cplx a[9], const cplx b[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            c[3 * i + j] = conj(a[i]) * b[j] + conj(a[3 + i]) * b[3 + j] + conj(a[6 + i]) * b[6 + j];
}

/* ------------------------------------------------------------------ */
/* Lattice geometry                                                    */
/* ------------------------------------------------------------------ */

typedef struct {
    int L[4];
    int64_t V;
} geom_t;

static inline void site_coords(const geom_t *g, int64_t s, int c[4])
{
    c[0] = (int)(s % g->L[0]);
    s /= g->L[0];
    c[1] = (int)(s % g->L[1]);
    s /= g->L[1];
    c[2] = (int)(s % g->L[2]);
    c[3] = (int)(s / g->L[2]);
}

static inline int64_t site_index(const geom_t *g, const int c[4])
{
    return (((int64_t)c[3] * g->L[2] + c[2]) * g->L[1] + c[1]) * g->L[0] + c[0];
}

static inline int64_t site_shift(const geom_t *g, int64_t s, int mu, int d)
{
    int c[4];
    site_coords(g, s, c);
    c[mu] = (c[mu] + d + g->L[mu]) % g->L[mu];
    return site_index(g, c);
}

/* Sum of the six staples around link U_mu(x), arranged so that
 * Re tr(U_mu(x) A) is the sum of Re tr over the plaquettes holding it:
 * A = sum_{nu != mu} [ U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
 *                    + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu) ]. */
static void staple(const geom_t *g, const cplx *U, int64_t x, int mu, cplx A[9])
{
    for (int i = 0; i < 9; ++i) A[i] = 0;
    int64_t xp = site_shift(g, x, mu, +1);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        int64_t xn = site_shift(g, x, nu, +1);
        int64_t xmn = site_shift(g, x, nu, -1);
        int64_t xpmn = site_shift(g, xp, nu, -1);
        cplx t1[9], t2[9];
        /* upper staple */
        mul33_nd(t1, U + 9 * (4 * xp + nu), U + 9 * (4 * xn + mu));
        mul33_nd(t2, t1, U + 9 * (4 * x + nu));
        for (int i = 0; i < 9; ++i) A[i] += t2[i];
        /* lower staple: U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu) */
        {
            cplx a[9];
            const cplx *un = U + 9 * (4 * xpmn + nu);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) a[3 * i + j] = conj(un[3 * j + i]);
            mul33_nd(t1, a, U + 9 * (4 * xmn + mu));
            mul33(t2, t1, U + 9 * (4 * xmn + nu));
        }
        for (int i = 0; i < 9; ++i) A[i] += t2[i];
    }
}

/* Average plaquette (1/3) Re tr U_P over all 6 V plaquettes. */
double dwfin_plaquette(const double *Ud, const int dims[4])
{
    geom_t g = {{dims[0], dims[1], dims[2], dims[3]}, (int64_t)dims[0] * dims[1] * dims[2] * dims[3]};
    const cplx *U = (const cplx *)Ud;
    double sum = 0.0;
#pragma omp parallel for reduction(+ : sum) schedule(static)
    for (int64_t x = 0; x < g.V; ++x) {
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                int64_t xm = site_shift(&g, x, mu, +1), xn = site_shift(&g, x, nu, +1);
                cplx a[9], b[9], c[9];
                mul33(a, U + 9 * (4 * x + mu), U + 9 * (4 * xm + nu));
                mul33_nd(b, a, U + 9 * (4 * xn + mu));
                mul33_nd(c, b, U + 9 * (4 * x + nu));
                sum += creal(c[0] + c[4] + c[8]) / 3.0;
            }
    }
    return sum / (6.0 * (double)g.V);
}

/* ------------------------------------------------------------------ */
/* SU(2) heatbath (Kennedy-Pendleton) inside SU(3) (Cabibbo-Marinari) */
/* ------------------------------------------------------------------ */

/* Draws h0 in [-1,1] with density proportional to sqrt(1-h0^2) exp(bp*h0)
 * by the Kennedy-Pendleton method: h0 = 1 - 2 lambda^2 where lambda^2 is a
 * Gamma(3/2, 2 bp) variate, accepted with probability sqrt(1 - lambda^2).
 * Random blocks come from counter (c0, c1, *draw, c3); *draw advances. */
static double kp_h0(double bp, const uint32_t key[2], uint32_t c0, uint32_t c1, uint32_t c3,
                    uint32_t *draw, int *ok)
{
    for (int tries = 0; tries < 100000; ++tries) {
        double u[2], v[2];
        uint32_t ctr[4] = {c0, c1, (*draw)++, c3};
        uniform2(ctr, key, u);
        ctr[2] = (*draw)++;
        uniform2(ctr, key, v);
        double cs = cos(6.283185307179586476925286766559 * u[1]);
        double lam2 = (-log(u[0]) - cs * cs * log(v[0])) / (2.0 * bp);
        if (v[1] * v[1] <= 1.0 - lam2) {
            *ok = 1;
            return 1.0 - 2.0 * lam2;
        }
    }
    *ok = 0;
    return 1.0;
}

/* Test hook: n samples of the Kennedy-Pendleton h0 at effective coupling bp. */
void dwfin_kp_samples(double *out, int64_t n, double bp, uint32_t seed)
{
    const uint32_t key[2] = {seed, 77u};
    for (int64_t i = 0; i < n; ++i) {
        uint32_t draw = 0;
        int ok;
        out[i] = kp_h0(bp, key, (uint32_t)i, 0u, (uint32_t)(i >> 32), &draw, &ok);
    }
}

static const int SUBGROUP[3][2] = {{0, 1}, {1, 2}, {0, 2}};

/* One Cabibbo-Marinari update of link U (3x3) given its staple sum A, at
 * gauge coupling beta, for action S = -(beta/3) sum_P Re tr U_P. */
static void cm_update(cplx Ul[9], const cplx A[9], double beta, const uint32_t key[2],
                      uint32_t c0, uint32_t c1base)
{
    for (int sg = 0; sg < 3; ++sg) {
        int i = SUBGROUP[sg][0], j = SUBGROUP[sg][1];
        cplx W[9];
        mul33(W, Ul, A);
        cplx w00 = W[3 * i + i], w01 = W[3 * i + j], w10 = W[3 * j + i], w11 = W[3 * j + j];
        /* Re tr(g w) = g . a for g = g0 + i g.sigma (g0+ig3, g2+ig1; -g2+ig1, g0-ig3) */
        double a[4];
        a[0] = creal(w00 + w11);
        a[1] = -cimag(w10 + w01);
        a[2] = creal(w10 - w01);
        a[3] = -cimag(w00 - w11);
        double k = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
        if (k < 1e-12) continue;
        double v[4] = {a[0] / k, a[1] / k, a[2] / k, a[3] / k};
        uint32_t draw = 0;
        int ok;
        uint32_t c1 = c1base + (uint32_t)sg;
        double h0 = kp_h0(beta * k / 3.0, key, c0, c1, 0u, &draw, &ok);
        if (!ok) continue;
        double u[2];
        uint32_t ctr[4] = {c0, c1, draw++, 0u};
        uniform2(ctr, key, u);
        double hr = sqrt(fmax(0.0, 1.0 - h0 * h0));
        double ct = 2.0 * u[0] - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct));
        double ph = 6.283185307179586476925286766559 * u[1];
        double h[4] = {h0, hr * st * cos(ph), hr * st * sin(ph), hr * ct};
        /* g = h V, quaternion product with V = v (as 2x2: v0+iv3, v2+iv1; -v2+iv1, v0-iv3) */
        cplx H2[4] = {h[0] + I * h[3], h[2] + I * h[1], -h[2] + I * h[1], h[0] - I * h[3]};
        cplx V2[4] = {v[0] + I * v[3], v[2] + I * v[1], -v[2] + I * v[1], v[0] - I * v[3]};
        cplx G2[4] = {H2[0] * V2[0] + H2[1] * V2[2], H2[0] * V2[1] + H2[1] * V2[3],
                      H2[2] * V2[0] + H2[3] * V2[2], H2[2] * V2[1] + H2[3] * V2[3]};
        /* U <- G U, G = embedding of G2 in rows/cols (i,j) */
        for (int c = 0; c < 3; ++c) {
            cplx ui = Ul[3 * i + c], uj = Ul[3 * j + c];
            Ul[3 * i + c] = G2[0] * ui + G2[1] * uj;
            Ul[3 * j + c] = G2[2] * ui + G2[3] * uj;
        }
    }
}

/* Random SU(3) matrices (hot start): Gram-Schmidt of Gaussian rows. */
void dwfin_random_su3(double *Ud, int64_t nmat, uint32_t seed, uint32_t stream)
{
    const uint32_t key[2] = {seed, stream};
    cplx *U = (cplx *)Ud;
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < nmat; ++m) {
        cplx *M = U + 9 * m;
        for (int e = 0; e < 6; ++e) {
            uint32_t ctr[4] = {(uint32_t)m, (uint32_t)e, 0u, (uint32_t)(m >> 32)};
            double gg[2];
            gauss2(ctr, key, gg);
            M[e] = gg[0] + I * gg[1];
        }
        M[6] = M[7] = M[8] = 0;
        dwfin_project_su3(M);
    }
}

/* Quenched heatbath: n_sweeps checkerboard Cabibbo-Marinari sweeps over
 * all links at coupling beta, starting from the links in U (modified in
 * place).  sweep_offset numbers the sweeps for the random stream, so that
 * a run split into pieces reproduces an unsplit run. */
int dwfin_heatbath(double *Ud, const int dims[4], double beta, int n_sweeps, int sweep_offset,
                   uint32_t seed)
{
    geom_t g = {{dims[0], dims[1], dims[2], dims[3]}, (int64_t)dims[0] * dims[1] * dims[2] * dims[3]};
    for (int mu = 0; mu < 4; ++mu)
        if (dims[mu] % 2) return -1; /* checkerboard needs even extents */
    cplx *U = (cplx *)Ud;
    const uint32_t key[2] = {seed, 0x48425448u /* "HBTH" */};
    for (int sw = 0; sw < n_sweeps; ++sw) {
        uint32_t sweep = (uint32_t)(sweep_offset + sw);
        for (int mu = 0; mu < 4; ++mu)
            for (int par = 0; par < 2; ++par) {
#pragma omp parallel for schedule(static)
                for (int64_t x = 0; x < g.V; ++x) {
                    int c[4];
                    site_coords(&g, x, c);
                    if (((c[0] + c[1] + c[2] + c[3]) & 1) != par) continue;
                    cplx A[9];
                    staple(&g, U, x, mu, A);
                    cm_update(U + 9 * (4 * x + mu), A, beta, key, (uint32_t)x,
                              (sweep * 4u + (uint32_t)mu) * 4u);
                    dwfin_project_su3(U + 9 * (4 * x + mu));
                }
            }
    }
    return 0;
}

int dwfin_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
