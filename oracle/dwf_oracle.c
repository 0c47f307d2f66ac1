/*
 * FP64 CPU oracle for the domain-wall fermion operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this code; it exists to check the GPU path.  It shares no
 * code, header, table or constant generator with the GPU path.
 *
 * The operator is the Shamir domain-wall operator of Cohen, Brower, Clark,
 * Osborn, "Multigrid Algorithms for Domain-Wall Fermions" (Sec. 2: the
 * operator has a fifth dimension of extent Ls whose walls carry the chiral
 * modes; Sec. 4: the fine operator couples each site to itself and its 10
 * unit-distance neighbours in five dimensions).  The paper does not write
 * the operator out; this file uses the standard unnormalised Shamir form:
 *
 *   (D psi)(x,s) = (5 - M5) psi(x,s)
 *       - 1/2 sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu,s)
 *                    + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu,s) ]
 *       - P_- psi(x,s+1) - P_+ psi(x,s-1)
 *   with the s = Ls-1 term  - P_- psi(x,Ls)  replaced by  + mf P_- psi(x,0)
 *   and  the s = 0    term  - P_+ psi(x,-1)  replaced by  + mf P_+ psi(x,Ls-1),
 *
 *   P_+- = (1 +- g_5)/2, gamma matrices in the chiral (DeGrand-Rossi) basis
 *   with g_5 = g_x g_y g_z g_t = diag(1,1,-1,-1).  Gauge links are periodic;
 *   the fermion is periodic in x,y,z and optionally antiperiodic in t (the
 *   hop across the t boundary picks up a factor -1).
 *
 * Fermion layout (canonical): f[((s*V + site)*4 + spin)*3 + colour],
 * site = ((t*Z + z)*Y + y)*X + x.  Links: U[((site*4 + mu)*3 + a)*3 + b].
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

/* gamma_mu, mu = 0..3 for x, y, z, t, in the DeGrand-Rossi chiral basis */
static const cplx GAMMA[4][4][4] = {
    /* gamma_x */
    {{0, 0, 0, I}, {0, 0, I, 0}, {0, -I, 0, 0}, {-I, 0, 0, 0}},
    /* gamma_y */
    {{0, 0, 0, -1}, {0, 0, 1, 0}, {0, 1, 0, 0}, {-1, 0, 0, 0}},
    /* gamma_z */
    {{0, 0, I, 0}, {0, 0, 0, -I}, {-I, 0, 0, 0}, {0, I, 0, 0}},
    /* gamma_t */
    {{0, 0, 1, 0}, {0, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, 0}},
};

/* gamma_5 diagonal: +1 on spins 0,1 (P_+), -1 on spins 2,3 (P_-) */
static const double GAMMA5[4] = {1.0, 1.0, -1.0, -1.0};

void orc_gamma(int mu, double *out /* 4x4 complex, row-major */)
{
    memcpy(out, GAMMA[mu], sizeof(GAMMA[mu]));
}

typedef struct {
    int L[4];
    int64_t V;
    int Ls;
    double M5, mf;
    int antiperiodic_t;
} lat_t;

static lat_t make_lat(const int dims[4], int Ls, double M5, double mf, int ap)
{
    lat_t l;
    for (int i = 0; i < 4; ++i) l.L[i] = dims[i];
    l.V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
    l.Ls = Ls;
    l.M5 = M5;
    l.mf = mf;
    l.antiperiodic_t = ap;
    return l;
}

static void coords(const lat_t *l, int64_t site, int c[4])
{
    c[0] = (int)(site % l->L[0]);
    site /= l->L[0];
    c[1] = (int)(site % l->L[1]);
    site /= l->L[1];
    c[2] = (int)(site % l->L[2]);
    c[3] = (int)(site / l->L[2]);
}

static int64_t index_of(const lat_t *l, const int c[4])
{
    return (((int64_t)c[3] * l->L[2] + c[2]) * l->L[1] + c[1]) * l->L[0] + c[0];
}

/* Neighbour x + d*mu (d = +1 or -1) and the boundary sign of the fermion. */
static int64_t neighbour(const lat_t *l, int64_t site, int mu, int d, double *sign)
{
    int c[4];
    coords(l, site, c);
    int n = c[mu] + d;
    *sign = 1.0;
    if (n == l->L[mu] || n == -1) {
        n = (n + l->L[mu]) % l->L[mu];
        if (mu == 3 && l->antiperiodic_t) *sign = -1.0;
    }
    c[mu] = n;
    return index_of(l, c);
}

static const cplx *spinor_at(const cplx *f, const lat_t *l, int s, int64_t site)
{
    return f + ((int64_t)s * l->V + site) * 12;
}

/* One hopping term, added into acc[4][3] (times `scale`):
 *   d = +1:  -1/2 (1 - g_mu) U_mu(x)          psi(x+mu)
 *   d = -1:  -1/2 (1 + g_mu) U_mu(x-mu)^dagger psi(x-mu)             */
static void add_hop(cplx acc[12], const cplx *in, const cplx *U, const lat_t *l, int s,
                    int64_t x, int mu, int d)
{
    double sign;
    int64_t y = neighbour(l, x, mu, d, &sign);
    const cplx *psi = spinor_at(in, l, s, y);
    cplx Upsi[4][3];
    if (d > 0) {
        const cplx *u = U + (x * 4 + mu) * 9;
        for (int sp = 0; sp < 4; ++sp)
            for (int a = 0; a < 3; ++a)
                Upsi[sp][a] = u[3 * a] * psi[3 * sp] + u[3 * a + 1] * psi[3 * sp + 1] +
                              u[3 * a + 2] * psi[3 * sp + 2];
    } else {
        const cplx *u = U + (y * 4 + mu) * 9;
        for (int sp = 0; sp < 4; ++sp)
            for (int a = 0; a < 3; ++a)
                Upsi[sp][a] = conj(u[a]) * psi[3 * sp] + conj(u[3 + a]) * psi[3 * sp + 1] +
                              conj(u[6 + a]) * psi[3 * sp + 2];
    }
    /* (1 - d*g_mu) applied in spin space */
    for (int sp = 0; sp < 4; ++sp)
        for (int a = 0; a < 3; ++a) {
            cplx v = Upsi[sp][a];
            for (int sq = 0; sq < 4; ++sq) v -= (double)d * GAMMA[mu][sp][sq] * Upsi[sq][a];
            acc[3 * sp + a] += -0.5 * sign * v;
        }
}

/* (D psi)(x, s) for one 5D site. */
static void D_site(cplx out[12], const cplx *in, const cplx *U, const lat_t *l, int s,
                   int64_t x)
{
    const cplx *p = spinor_at(in, l, s, x);
    for (int i = 0; i < 12; ++i) out[i] = (5.0 - l->M5) * p[i];
    for (int mu = 0; mu < 4; ++mu) {
        add_hop(out, in, U, l, s, x, mu, +1);
        add_hop(out, in, U, l, s, x, mu, -1);
    }
    /* fifth-dimension hops: -P_- psi(s+1) and -P_+ psi(s-1); at the walls
     * they wrap with coefficient +mf instead of -1. */
    {
        int sn = (s == l->Ls - 1) ? 0 : s + 1;
        double c = (s == l->Ls - 1) ? l->mf : -1.0;
        const cplx *q = spinor_at(in, l, sn, x);
        for (int sp = 2; sp < 4; ++sp) /* P_- keeps spins 2,3 */
            for (int a = 0; a < 3; ++a) out[3 * sp + a] += c * q[3 * sp + a];
    }
    {
        int sn = (s == 0) ? l->Ls - 1 : s - 1;
        double c = (s == 0) ? l->mf : -1.0;
        const cplx *q = spinor_at(in, l, sn, x);
        for (int sp = 0; sp < 2; ++sp) /* P_+ keeps spins 0,1 */
            for (int a = 0; a < 3; ++a) out[3 * sp + a] += c * q[3 * sp + a];
    }
}

void orc_apply_D(double *out_, const double *in_, const double *U_, const int dims[4], int Ls,
                 double M5, double mf, int antiperiodic_t)
{
    lat_t l = make_lat(dims, Ls, M5, mf, antiperiodic_t);
    cplx *out = (cplx *)out_;
    const cplx *in = (const cplx *)in_, *U = (const cplx *)U_;
    int64_t n5 = l.V * Ls;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n5; ++i) {
        int s = (int)(i / l.V);
        int64_t x = i % l.V;
        D_site(out + i * 12, in, U, &l, s, x);
    }
}

/* (D psi) at a list of 5D sites idx5[k] = s*V + site; out is [n][12]. */
void orc_apply_D_sites(double *out_, const double *in_, const double *U_, const int dims[4],
                       int Ls, double M5, double mf, int antiperiodic_t, const int64_t *idx5,
                       int64_t n)
{
    lat_t l = make_lat(dims, Ls, M5, mf, antiperiodic_t);
    cplx *out = (cplx *)out_;
    const cplx *in = (const cplx *)in_, *U = (const cplx *)U_;
    for (int64_t k = 0; k < n; ++k)
        D_site(out + k * 12, in, U, &l, (int)(idx5[k] / l.V), idx5[k] % l.V);
}

/* Gamma = gamma_5 R_5 with (R_5 psi)(s) = psi(Ls-1-s). */
static void apply_Gamma(cplx *out, const cplx *in, const lat_t *l)
{
    for (int s = 0; s < l->Ls; ++s)
        for (int64_t x = 0; x < l->V; ++x) {
            const cplx *p = spinor_at(in, l, l->Ls - 1 - s, x);
            cplx *o = out + ((int64_t)s * l->V + x) * 12;
            for (int sp = 0; sp < 4; ++sp)
                for (int a = 0; a < 3; ++a) o[3 * sp + a] = GAMMA5[sp] * p[3 * sp + a];
        }
}

/* D^dagger = Gamma D Gamma (the gamma_5 R_5 hermiticity of the Shamir operator). */
void orc_apply_Ddag(double *out_, const double *in_, const double *U_, const int dims[4],
                    int Ls, double M5, double mf, int antiperiodic_t)
{
    lat_t l = make_lat(dims, Ls, M5, mf, antiperiodic_t);
    int64_t n = l.V * Ls * 12;
    cplx *t1 = malloc(sizeof(cplx) * n), *t2 = malloc(sizeof(cplx) * n);
    apply_Gamma(t1, (const cplx *)in_, &l);
    orc_apply_D((double *)t2, (const double *)t1, U_, dims, Ls, M5, mf, antiperiodic_t);
    apply_Gamma((cplx *)out_, t2, &l);
    free(t1);
    free(t2);
}

/* One hopping term alone over the whole lattice:
 *   out(x,s) = -1/2 (1 - d g_mu) U^(d)(x) in(x + d mu, s). */
void orc_hop(double *out_, const double *in_, const double *U_, const int dims[4], int Ls,
             int mu, int d, int antiperiodic_t)
{
    lat_t l = make_lat(dims, Ls, 0.0, 0.0, antiperiodic_t);
    cplx *out = (cplx *)out_;
    const cplx *in = (const cplx *)in_, *U = (const cplx *)U_;
    int64_t n5 = l.V * Ls;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n5; ++i) {
        cplx acc[12] = {0};
        add_hop(acc, in, U, &l, (int)(i / l.V), i % l.V, mu, d);
        memcpy(out + i * 12, acc, sizeof(acc));
    }
}
