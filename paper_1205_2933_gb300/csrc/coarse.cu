// The Galerkin coarse operator R A P (Sec. 2, third step of the V-cycle:
// S2 acts on R A P) as a 9-point stencil of dense n x n complex blocks:
//   (A_c c)(x) = Y0(x) c(x) + sum_{mu, dir} Y_{mu,dir}(x) c(x + dir*mu),
// direction index d = 0 (self), 1 + 2*mu (+mu), 2 + 2*mu (-mu); storage
// Y[x][d][k][l].  One fine hop crosses at most one block face, so the
// unsquared operator coarsens to nearest neighbours (Sec. 4 contrasts this
// with the squared operator's two-hop coarse stencil, which has 33 points
// when every block extent is at least 2).
//
// Construction (FP64): with q_l the block-orthonormal basis,
//   Y_{mu,dir}(x)[k][l] = sum over the sites of block x whose hop along
//                         dir*mu leaves the block of conj(q_k) . hop(q_l),
//   Y0(x)[k][l]         = <q_k, A q_l>_block - sum_{mu,dir} Y_{mu,dir}(x)[k][l].
#include "mg.cuh"
#include "spin.cuh"

#include <type_traits>

namespace dwf {

namespace {

template <typename LT> struct LinkRead;
template <> struct LinkRead<double2> {
    template <typename R> static __device__ __forceinline__ C<R> get(const double2 *Y, int64_t i) { return cvt<C<R>, double2>(Y[i]); }
};
template <> struct LinkRead<float2> {
    template <typename R> static __device__ __forceinline__ C<R> get(const float2 *Y, int64_t i) { return cvt<C<R>, float2>(Y[i]); }
};
template <> struct LinkRead<__nv_bfloat162> {
    template <typename R> static __device__ __forceinline__ C<R> get(const __nv_bfloat162 *Y, int64_t i) {
        float2 f = __bfloat1622float2(Y[i]);
        return cvt<C<R>, float2>(f);
    }
};
template <> struct LinkRead<__half2> {
    template <typename R> static __device__ __forceinline__ C<R> get(const __half2 *Y, int64_t i) {
        float2 f = __half22float2(Y[i]);
        return cvt<C<R>, float2>(f);
    }
};

__device__ __forceinline__ int64_t shift_site(const Geom &g, int64_t site, int mu, int dir) {
    int c[4];
    site_coords(g, site, c);
    c[mu] += dir;
    if (c[mu] == g.L[mu]) c[mu] = 0;
    if (c[mu] < 0) c[mu] = g.L[mu] - 1;
    return site_index(g, c);
}

template <typename R, typename LT, int NV, bool DAG, int NPTS>
__global__ void __launch_bounds__(256) coarse_apply_kernel(C<R> *__restrict__ y, const C<R> *__restrict__ x,
                                                           const LT *__restrict__ Y, Geom g,
                                                           const int *__restrict__ nbr) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t field = g.V * NV;
    if (i >= field) return;
    x += blockIdx.y * field;
    y += blockIdx.y * field;
    const int64_t site = i / NV;
    const int k = (int)(i - site * NV);
    C<R> acc = mk<R>(0, 0);
#pragma unroll 1
    for (int d = 0; d < NPTS; ++d) {
        int64_t other = site;
        // table entry 2 mu: +mu, 2 mu + 1: -mu; D^+ reads the opposite neighbour
        // (9 points only: the 33-point stencil is Hermitian)
        if (d > 0) other = nbr[site * (NPTS - 1) + (DAG ? ((d - 1) ^ 1) : (d - 1))];
        const C<R> *xv = x + other * NV;
        if (!DAG) {
            const int64_t row = ((site * NPTS + d) * NV + k) * NV;
#pragma unroll 8
            for (int l = 0; l < NV; ++l) cfma(acc, LinkRead<LT>::template get<R>(Y, row + l), xv[l]);
        } else {
            const int64_t base = (other * NPTS + d) * NV * NV + k;
#pragma unroll 8
            for (int l = 0; l < NV; ++l) cfmac(acc, LinkRead<LT>::template get<R>(Y, base + (int64_t)l * NV), xv[l]);
        }
    }
    y[i] = acc;
}

// ---- construction -------------------------------------------------------

struct FaceMap {
    int L[4], b[4], Lc[4];
    int Ls;      // fifth extent of the finer level (1 on coarse levels)
    int run;     // components per face element (12 fine, n coarse)
    int64_t nelem;
};

// 4D coordinates of face site f (0 <= f < bsites/b_mu * Ls) of block xc for (mu, dir)
__device__ __forceinline__ void face_site(const FaceMap &m, int64_t xc, int mu, int dir, int64_t f, int64_t &site,
                                          int &s) {
    s = (int)(f % m.Ls);
    int64_t i = f / m.Ls;
    int c[4], o[4];
    int64_t t = xc;
    c[0] = (int)(t % m.Lc[0]); t /= m.Lc[0];
    c[1] = (int)(t % m.Lc[1]); t /= m.Lc[1];
    c[2] = (int)(t % m.Lc[2]); c[3] = (int)(t / m.Lc[2]);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) {
            o[nu] = dir > 0 ? m.b[nu] - 1 : 0;
        } else {
            o[nu] = (int)(i % m.b[nu]);
            i /= m.b[nu];
        }
    }
    site = (((int64_t)(c[3] * m.b[3] + o[3]) * m.L[2] + (c[2] * m.b[2] + o[2])) * m.L[1] + (c[1] * m.b[1] + o[1])) *
               m.L[0] + (c[0] * m.b[0] + o[0]);
}

// The hop of the fine D from x = site (fifth coordinate s) to x + dir*mu,
// -1/2 (1 -+ gamma_mu) U q(x +- mu) with the antiperiodic sign in t.
template <typename R>
__device__ __forceinline__ void fine_face_hop(C<R> acc12[12], const C<R> *ql, const C<R> *U, const Geom &g, int Ls,
                                              int64_t site, int s, int mu, int dir) {
    int c[4];
    site_coords(g, site, c);
    int cc[4] = {c[0], c[1], c[2], c[3]};
    cc[mu] += dir;
    bool wrap = (cc[mu] == g.L[mu] || cc[mu] < 0);
    if (cc[mu] == g.L[mu]) cc[mu] = 0;
    if (cc[mu] < 0) cc[mu] = g.L[mu] - 1;
    int64_t nb = site_index(g, cc);
    R coef = (mu == 3 && g.ap && wrap) ? R(0.5) : R(-0.5);
    for (int e = 0; e < 12; ++e) acc12[e] = mk<R>(0, 0);
    C<R> lk[9];
    LinkIO<R>::load(U, dir > 0 ? site : nb, mu, lk);
    if (dir > 0) {
        switch (mu) {
            case 0: hop<0, false, R>(acc12, ql, nb, Ls, s, lk, -1, coef); break;
            case 1: hop<1, false, R>(acc12, ql, nb, Ls, s, lk, -1, coef); break;
            case 2: hop<2, false, R>(acc12, ql, nb, Ls, s, lk, -1, coef); break;
            default: hop<3, false, R>(acc12, ql, nb, Ls, s, lk, -1, coef); break;
        }
    } else {
        switch (mu) {
            case 0: hop<0, true, R>(acc12, ql, nb, Ls, s, lk, +1, coef); break;
            case 1: hop<1, true, R>(acc12, ql, nb, Ls, s, lk, +1, coef); break;
            case 2: hop<2, true, R>(acc12, ql, nb, Ls, s, lk, +1, coef); break;
            default: hop<3, true, R>(acc12, ql, nb, Ls, s, lk, +1, coef); break;
        }
    }
}

// F[xc][dd][k][l], dd = 2*mu + (dir < 0): block-face contributions of one hop.
// FINE: hop = -1/2 (1 -+ g_mu) U q_l(x +- mu) with boundary sign (the fine D);
// else: hop = Y_d(x) q_l(x +- mu) of the finer coarse level's stencil.
template <int NV, bool FINE, typename R>
__global__ void __launch_bounds__(256) face_kernel(double2 *__restrict__ F, const C<R> *__restrict__ Q,
                                                   const C<R> *__restrict__ U, const double2 *__restrict__ Yf,
                                                   Geom g, FaceMap m, int chf) {
    extern __shared__ unsigned char sm_raw[];
    C<R> *sm = reinterpret_cast<C<R> *>(sm_raw);
    const int run = m.run;
    C<R> *sH = sm;                        // [NV][chf*run]
    C<R> *sA = sm + (size_t)NV * chf * run;  // [NV][chf*run]
    const int64_t xc = blockIdx.x;
    const int dd = blockIdx.y;
    const int mu = dd >> 1, dir = (dd & 1) ? -1 : +1;
    const int64_t nface = (int64_t)m.b[0] * m.b[1] * m.b[2] * m.b[3] / m.b[mu] * m.Ls;
    constexpr int NP = NV * NV;
    constexpr int PPT = (NP + 255) / 256;
    double2 acc[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) acc[q] = make_double2(0, 0);
    const int W = chf * run;
    for (int64_t f0 = 0; f0 < nface; f0 += chf) {
        // hops of every q_l at the chunk's face sites, and q_k there
        for (int item = threadIdx.x; item < NV * chf; item += blockDim.x) {
            int l = item / chf, fl = item - l * chf;
            int64_t f = f0 + fl;
            C<R> *h = sH + (size_t)l * W + fl * run;
            C<R> *a = sA + (size_t)l * W + fl * run;
            if (f >= nface) {
                for (int e = 0; e < run; ++e) { h[e] = mk<R>(0, 0); a[e] = mk<R>(0, 0); }
                continue;
            }
            int64_t site;
            int s;
            face_site(m, xc, mu, dir, f, site, s);
            const C<R> *ql = Q + (int64_t)l * m.nelem;
            if (FINE) {
                for (int e = 0; e < 12; ++e) a[e] = ql[(site * 12 + e) * m.Ls + s];
                C<R> acc12[12];
                fine_face_hop<R>(acc12, ql, U, g, m.Ls, site, s, mu, dir);
                for (int e = 0; e < 12; ++e) h[e] = acc12[e];
            } else {
                for (int e = 0; e < run; ++e) a[e] = ql[site * run + e];
                int64_t nb = shift_site(g, site, mu, dir);
                const double2 *Yrow = Yf + (site * 9 + 1 + dd) * (int64_t)run * run;
                const C<R> *qn = ql + nb * run;
                for (int e = 0; e < run; ++e) {
                    C<R> z = mk<R>(0, 0);
                    for (int m2 = 0; m2 < run; ++m2) cfma(z, cvt<C<R>, double2>(Yrow[e * run + m2]), qn[m2]);
                    h[e] = z;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            int p = threadIdx.x + q * 256;
            if (p < NP) {
                int k = p / NV, l = p - k * NV;
                const C<R> *ak = sA + (size_t)k * W, *hl = sH + (size_t)l * W;
                C<R> s = mk<R>(0, 0);
                for (int e = 0; e < W; ++e) cfmac(s, ak[e], hl[e]);
                acc[q].x += (double)s.x;
                acc[q].y += (double)s.y;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        int p = threadIdx.x + q * 256;
        if (p < NP) F[(xc * 8 + dd) * NP + p] = acc[q];
    }
}

__global__ void assemble_kernel(double2 *__restrict__ Y, const double2 *__restrict__ G0, const double2 *__restrict__ F,
                                int64_t nc, int nv) {
    const int64_t np = (int64_t)nv * nv;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc * np; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t xc = i / np, p = i - xc * np;
        double2 y0 = G0[i];
        for (int dd = 0; dd < 8; ++dd) {
            double2 f = F[(xc * 8 + dd) * np + p];
            Y[(xc * 9 + 1 + dd) * np + p] = f;
            y0.x -= f.x;
            y0.y -= f.y;
        }
        Y[(xc * 9) * np + p] = y0;
    }
}

template <typename TO>
__global__ void convert_kernel(TO *__restrict__ out, const double2 *__restrict__ in, int64_t n);
template <>
__global__ void convert_kernel<float2>(float2 *__restrict__ out, const double2 *__restrict__ in, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
template <>
__global__ void convert_kernel<__nv_bfloat162>(__nv_bfloat162 *__restrict__ out, const double2 *__restrict__ in, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __floats2bfloat162_rn((float)in[i].x, (float)in[i].y);
}
template <>
__global__ void convert_kernel<__half2>(__half2 *__restrict__ out, const double2 *__restrict__ in, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __floats2half2_rn((float)in[i].x, (float)in[i].y);
}

#define NV_DISPATCH2(nv, MACRO)                                     \
    switch (nv) {                                                   \
        case 2: MACRO(2); break;                                    \
        case 4: MACRO(4); break;                                    \
        case 6: MACRO(6); break;                                    \
        case 8: MACRO(8); break;                                    \
        case 12: MACRO(12); break;                                  \
        case 16: MACRO(16); break;                                  \
        case 24: MACRO(24); break;                                  \
        case 32: MACRO(32); break;                                  \
        default: throw Error{DWF_EINVAL, "unsupported Nvec (use 2,4,6,8,12,16,24,32)"}; \
    }

template <typename R, typename LT>
void coarse_apply_t(dwf_ctx *c, const Level &L, C<R> *y, const C<R> *x, const LT *Y, bool dag, int nrhs) {
    const Geom &g = L.lg.g;
    int n = L.lg.ncomp;
    const int *nbrt = L.nbr.as<int>();
    DWF_REQUIRE(nbrt, DWF_ESTATE, "coarse level without a neighbour table");
    dim3 grid((unsigned)((g.V * n + 255) / 256), (unsigned)nrhs);
#define CK(NV)                                                                                               \
    if (L.npts == 33) coarse_apply_kernel<R, LT, NV, false, 33><<<grid, 256, 0, c->stream>>>(y, x, Y, g, nbrt); \
    else if (dag) coarse_apply_kernel<R, LT, NV, true, 9><<<grid, 256, 0, c->stream>>>(y, x, Y, g, nbrt);    \
    else coarse_apply_kernel<R, LT, NV, false, 9><<<grid, 256, 0, c->stream>>>(y, x, Y, g, nbrt)
    NV_DISPATCH2(n, CK);
#undef CK
    DWF_CHECK_LAUNCH();
}

}  // namespace

template <typename R> void coarse_apply(dwf_ctx *c, const Level &L, C<R> *y, const C<R> *x, bool dag) {
    ProfScope ps(c, K_COARSE);
    switch (L.yprec) {
        case DWF_F64: coarse_apply_t<R, double2>(c, L, y, x, L.Y64.as<double2>(), dag, 1); break;
        case DWF_F32: coarse_apply_t<R, float2>(c, L, y, x, L.Y32.as<float2>(), dag, 1); break;
        case DWF_BF16: coarse_apply_t<R, __nv_bfloat162>(c, L, y, x, L.Y16.as<__nv_bfloat162>(), dag, 1); break;
        case DWF_F16: coarse_apply_t<R, __half2>(c, L, y, x, L.Y16.as<__half2>(), dag, 1); break;
    }
}

void convert_coarse_links(dwf_ctx *c, Level &L) {
    int64_t n = L.lg.g.V * L.npts * (int64_t)L.lg.ncomp * L.lg.ncomp;
    unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 16);
    if (L.yprec == DWF_F32) {
        if (L.Y32.bytes < sizeof(float2) * n) L.Y32.alloc(sizeof(float2) * n);
        convert_kernel<float2><<<blocks, 256, 0, c->stream>>>(L.Y32.as<float2>(), L.Y64.as<double2>(), n);
    } else if (L.yprec == DWF_BF16) {
        if (L.Y16.bytes < 4 * n) L.Y16.alloc(4 * n);
        convert_kernel<__nv_bfloat162><<<blocks, 256, 0, c->stream>>>(L.Y16.as<__nv_bfloat162>(), L.Y64.as<double2>(), n);
    } else if (L.yprec == DWF_F16) {
        if (L.Y16.bytes < 4 * n) L.Y16.alloc(4 * n);
        convert_kernel<__half2><<<blocks, 256, 0, c->stream>>>(L.Y16.as<__half2>(), L.Y64.as<double2>(), n);
    }
    DWF_CHECK_LAUNCH();
    build_tc_images(c, L);
}

// Build Y of level Lc = L+1 (FP64) from level L's basis Q in precision R:
// FP32 products with FP64 accumulation across chunks when R = float.
template <typename R> void build_coarse_from(dwf_ctx *c, Level &L, Level &Lc, const C<R> *Q, C<R> *W) {
    const int nv = L.nv;
    // W_l = A_l q_l for every basis vector
    if (L.index == 0) {
        dslash(c, W, Q, false, nv);
    } else {
        for (int l = 0; l < nv; ++l)
            coarse_apply_t<R, double2>(c, L, W + (int64_t)l * L.lg.nelem, Q + (int64_t)l * L.lg.nelem,
                                       L.Y64.as<double2>(), false, 1);
    }
    const int64_t nc = Lc.lg.g.V;
    const int64_t np = (int64_t)nv * nv;
    if (L.G.bytes < sizeof(double2) * nc * np) L.G.alloc(sizeof(double2) * nc * np);
    if (L.F.bytes < sizeof(double2) * nc * np * 8) L.F.alloc(sizeof(double2) * nc * np * 8);
    block_gram<R>(c, L, L.G.as<double2>(), Q, W);
    FaceMap m;
    for (int i = 0; i < 4; ++i) {
        m.L[i] = L.lg.g.L[i];
        m.b[i] = L.block[i];
        m.Lc[i] = m.L[i] / m.b[i];
    }
    m.Ls = L.lg.g.Ls;
    m.run = L.lg.ncomp;
    m.nelem = L.lg.nelem;
    int chf = (int)std::max<int64_t>(1, (46 * 1024) / ((int64_t)2 * nv * m.run * sizeof(C<R>)));
    size_t smem = (size_t)2 * nv * chf * m.run * sizeof(C<R>);
    dim3 grid((unsigned)nc, 8);
    bool fine = (L.index == 0);
    const C<R> *Ul = std::is_same<R, double>::value ? (const C<R> *)c->U64.p : (const C<R> *)c->U32.p;
#define FK(NV)                                                                                               \
    if (fine) face_kernel<NV, true, R><<<grid, 256, smem, c->stream>>>(L.F.as<double2>(), Q, Ul, nullptr,     \
                                                                      L.lg.g, m, chf);                       \
    else face_kernel<NV, false, R><<<grid, 256, smem, c->stream>>>(L.F.as<double2>(), Q, nullptr,            \
                                                                  L.Y64.as<double2>(), L.lg.g, m, chf)
    NV_DISPATCH2(nv, FK);
#undef FK
    DWF_CHECK_LAUNCH();
    size_t yb = sizeof(double2) * nc * 9 * np;
    if (Lc.Y64.bytes < yb) Lc.Y64.alloc(yb);
    unsigned blocks = (unsigned)std::min<int64_t>((nc * np + 255) / 256, (int64_t)c->sm_count * 16);
    assemble_kernel<<<blocks, 256, 0, c->stream>>>(Lc.Y64.as<double2>(), L.G.as<double2>(), L.F.as<double2>(), nc, nv);
    DWF_CHECK_LAUNCH();
    convert_coarse_links(c, Lc);
}

// ---- the squared operator's coarse stencil (Sec. 4) -----------------------
//
// P^+ D^+ D P as 33 dense n x n blocks per coarse site.  D q_l splits by
// where its terms read q_l: T_0 (diagonal, fifth-dimension hops, hops inside
// the block of x) and T_sigma for the 8 hops x -> x + dir mu that leave the
// block (sigma = 1 + 2 mu for dir = +1, 2 + 2 mu for dir = -1, supported on
// the block's last resp. first layer in mu).  On block b'', D applied to the
// basis piece of block b' = b'' + sigma is T_sigma there, so
//   Y[b''+sigma1][sigma2 - sigma1][k][l] += <T_{sigma1,k}, T_{sigma2,l}>_{b''}
// summed over b'' and the 73 pairs (sigma1, sigma2) whose supports meet
// (the pairs +mu/-mu never do when every block extent is >= 2).

namespace {

constexpr int SQ_PAIRS = 73;

struct PairTable {
    int s1[SQ_PAIRS], s2[SQ_PAIRS], d[SQ_PAIRS];  // source offsets (0..8) and stencil index (0..32)
};

void sigma_vec(int sg, int v[4]) {
    for (int i = 0; i < 4; ++i) v[i] = 0;
    if (sg > 0) v[(sg - 1) >> 1] = ((sg - 1) & 1) ? -1 : +1;
}

PairTable make_pairs() {
    int off[33][4];
    squared_offsets(off);
    PairTable t;
    int n = 0;
    for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b) {
            int va[4], vb[4], dv[4];
            sigma_vec(a, va);
            sigma_vec(b, vb);
            for (int i = 0; i < 4; ++i) dv[i] = vb[i] - va[i];
            int idx = -1;
            for (int d = 0; d < 33 && idx < 0; ++d)
                if (off[d][0] == dv[0] && off[d][1] == dv[1] && off[d][2] == dv[2] && off[d][3] == dv[3]) idx = d;
            if (idx < 0) continue;  // +-2 mu
            t.s1[n] = a;
            t.s2[n] = b;
            t.d[n] = idx;
            ++n;
        }
    if (n != SQ_PAIRS) throw Error{DWF_ECUDA, "squared coarse stencil: pair table size"};
    return t;
}

// face element f = i*Ls + s of block xc for (mu, dir): its fine site
__device__ __forceinline__ int64_t face_elem_site(const FaceMap &m, int64_t xc, int mu, int dir, int64_t f, int &s) {
    int64_t site;
    face_site(m, xc, mu, dir, f, site, s);
    return site;
}

// Hf[dd][l][xc][(i*12 + e)*Ls + s] = T_{1+dd}(q_l) at face element (i, s) of block xc
template <typename R>
__global__ void __launch_bounds__(256) face_terms_kernel(C<R> *__restrict__ Hf, const C<R> *__restrict__ Q,
                                                         const C<R> *__restrict__ U, Geom g, FaceMap m, int64_t nc,
                                                         int64_t nfe) {
    const int64_t xc = blockIdx.x;
    const int dd = blockIdx.y, l = blockIdx.z;
    const int mu = dd >> 1, dir = (dd & 1) ? -1 : +1;
    const int nv = gridDim.z;
    const int64_t nface = (int64_t)m.b[0] * m.b[1] * m.b[2] * m.b[3] / m.b[mu] * m.Ls;
    const C<R> *ql = Q + (int64_t)l * m.nelem;
    C<R> *out = Hf + (((int64_t)dd * nv + l) * nc + xc) * nfe;
    for (int64_t f = threadIdx.x; f < nface; f += blockDim.x) {
        int s;
        const int64_t site = face_elem_site(m, xc, mu, dir, f, s);
        C<R> h[12];
        fine_face_hop<R>(h, ql, U, g, m.Ls, site, s, mu, dir);
        const int64_t i = f / m.Ls;
        for (int e = 0; e < 12; ++e) out[(i * 12 + e) * m.Ls + s] = h[e];
    }
}

// W_l -= T_{1+dd}(q_l) on the face of every block (one dd per launch: no two
// threads of a launch touch the same element)
template <typename R>
__global__ void __launch_bounds__(256) subtract_faces_kernel(C<R> *__restrict__ W, const C<R> *__restrict__ Hf,
                                                             FaceMap m, int64_t nc, int64_t nfe, int dd) {
    const int64_t xc = blockIdx.x;
    const int l = blockIdx.y, nv = gridDim.y;
    const int mu = dd >> 1, dir = (dd & 1) ? -1 : +1;
    const int64_t nface = (int64_t)m.b[0] * m.b[1] * m.b[2] * m.b[3] / m.b[mu] * m.Ls;
    const C<R> *h = Hf + (((int64_t)dd * nv + l) * nc + xc) * nfe;
    C<R> *w = W + (int64_t)l * m.nelem;
    for (int64_t f = threadIdx.x; f < nface; f += blockDim.x) {
        int s;
        const int64_t site = face_elem_site(m, xc, mu, dir, f, s);
        const int64_t i = f / m.Ls;
        for (int e = 0; e < 12; ++e) {
            C<R> v = w[(site * 12 + e) * m.Ls + s];
            const C<R> t = h[(i * 12 + e) * m.Ls + s];
            v.x -= t.x;
            v.y -= t.y;
            w[(site * 12 + e) * m.Ls + s] = v;
        }
    }
}

// T_sg(q_l) at block-local coordinates o, component e, fifth coordinate s of block xc
template <typename R>
__device__ __forceinline__ C<R> t_value(const C<R> *W, const C<R> *Hf, const FaceMap &m, int64_t xc, const int xcc[4],
                                        int sg, int l, int nv, int64_t nc, int64_t nfe, const int o[4], int e, int s) {
    if (sg == 0) {
        const int64_t site = (((int64_t)(xcc[3] * m.b[3] + o[3]) * m.L[2] + (xcc[2] * m.b[2] + o[2])) * m.L[1] +
                              (xcc[1] * m.b[1] + o[1])) * m.L[0] + (xcc[0] * m.b[0] + o[0]);
        return W[(int64_t)l * m.nelem + (site * 12 + e) * m.Ls + s];
    }
    const int dd = sg - 1, mu = dd >> 1;
    int64_t i = 0, stride = 1;
    for (int nu = 0; nu < 4; ++nu)
        if (nu != mu) {
            i += o[nu] * stride;
            stride *= m.b[nu];
        }
    return Hf[(((int64_t)dd * nv + l) * nc + xc) * nfe + (i * 12 + e) * m.Ls + s];
}

// Gp[xc][p][k][l] = <T_{s1(p),k}, T_{s2(p),l}> over the sites of block xc
// where both are supported (FP64 accumulation across chunks of ch elements)
template <int NV, typename R>
__global__ void __launch_bounds__(256) pair_gram_kernel(double2 *__restrict__ Gp, const C<R> *__restrict__ W,
                                                        const C<R> *__restrict__ Hf, FaceMap m, PairTable pt,
                                                        int64_t nc, int64_t nfe, int ch) {
    extern __shared__ unsigned char sm_raw[];
    C<R> *sA = reinterpret_cast<C<R> *>(sm_raw);  // [NV][ch]
    C<R> *sB = sA + (size_t)NV * ch;              // [NV][ch]
    const int64_t xc = blockIdx.x;
    const int p = blockIdx.y;
    const int s1 = pt.s1[p], s2 = pt.s2[p];
    int xcc[4];
    {
        int64_t t = xc;
        xcc[0] = (int)(t % m.Lc[0]); t /= m.Lc[0];
        xcc[1] = (int)(t % m.Lc[1]); t /= m.Lc[1];
        xcc[2] = (int)(t % m.Lc[2]); xcc[3] = (int)(t / m.Lc[2]);
    }
    // the region where both pieces live: a box inside the block
    int lo[4], ext[4];
    for (int nu = 0; nu < 4; ++nu) { lo[nu] = 0; ext[nu] = m.b[nu]; }
    const int sgs[2] = {s1, s2};
    for (int j = 0; j < 2; ++j)
        if (const int sg = sgs[j]; sg > 0) {
            const int mu = (sg - 1) >> 1;
            lo[mu] = ((sg - 1) & 1) ? 0 : m.b[mu] - 1;
            ext[mu] = 1;
        }
    const int64_t nel = (int64_t)ext[0] * ext[1] * ext[2] * ext[3] * 12 * m.Ls;
    constexpr int NP = NV * NV;
    constexpr int PPT = (NP + 255) / 256;
    double2 acc[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) acc[q] = make_double2(0, 0);
    for (int64_t e0 = 0; e0 < nel; e0 += ch) {
        for (int item = threadIdx.x; item < NV * ch; item += blockDim.x) {
            const int l = item / ch, fl = item - l * ch;
            const int64_t r = e0 + fl;
            C<R> a = mk<R>(0, 0), b = mk<R>(0, 0);
            if (r < nel) {
                const int s = (int)(r % m.Ls);
                int64_t t = r / m.Ls;
                const int e = (int)(t % 12);
                t /= 12;
                int o[4];
                for (int nu = 0; nu < 4; ++nu) {
                    o[nu] = lo[nu] + (int)(t % ext[nu]);
                    t /= ext[nu];
                }
                a = t_value<R>(W, Hf, m, xc, xcc, s1, l, NV, nc, nfe, o, e, s);
                b = t_value<R>(W, Hf, m, xc, xcc, s2, l, NV, nc, nfe, o, e, s);
            }
            sA[(size_t)l * ch + fl] = a;
            sB[(size_t)l * ch + fl] = b;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const int pp = threadIdx.x + q * 256;
            if (pp < NP) {
                const int k = pp / NV, l = pp - k * NV;
                const C<R> *ak = sA + (size_t)k * ch, *bl = sB + (size_t)l * ch;
                C<R> sum = mk<R>(0, 0);
                for (int e = 0; e < ch; ++e) cfmac(sum, ak[e], bl[e]);
                acc[q].x += (double)sum.x;
                acc[q].y += (double)sum.y;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int pp = threadIdx.x + q * 256;
        if (pp < NP) Gp[((int64_t)xc * SQ_PAIRS + p) * NP + pp] = acc[q];
    }
}

// Y[b][d][k][l] = sum over pairs p with stencil index d of Gp[b - sigma1(p)][p][k][l],
// pairs in a fixed order (deterministic)
__global__ void assemble_squared_kernel(double2 *__restrict__ Y, const double2 *__restrict__ Gp, Geom gc,
                                        PairTable pt, int nv) {
    const int64_t np = (int64_t)nv * nv;
    const int64_t total = gc.V * 33 * np;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / (33 * np);
        const int d = (int)((i / np) % 33);
        const int64_t kk = i % np;
        int cb[4];
        site_coords(gc, b, cb);
        double2 y = make_double2(0, 0);
        for (int p = 0; p < SQ_PAIRS; ++p) {
            if (pt.d[p] != d) continue;
            int cc[4] = {cb[0], cb[1], cb[2], cb[3]};
            const int sg = pt.s1[p];
            if (sg > 0) {
                const int mu = (sg - 1) >> 1, dir = ((sg - 1) & 1) ? -1 : +1;
                cc[mu] = (cc[mu] - dir + gc.L[mu]) % gc.L[mu];
            }
            const double2 g = Gp[(site_index(gc, cc) * SQ_PAIRS + p) * np + kk];
            y.x += g.x;
            y.y += g.y;
        }
        Y[i] = y;
    }
}

}  // namespace

void squared_offsets(int off[33][4]) {
    for (int d = 0; d < 33; ++d)
        for (int i = 0; i < 4; ++i) off[d][i] = 0;
    for (int mu = 0; mu < 4; ++mu) {
        off[1 + 2 * mu][mu] = +1;
        off[2 + 2 * mu][mu] = -1;
    }
    static const int pairs[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    for (int p = 0; p < 6; ++p)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const int d = 9 + 4 * p + 2 * a + b;
                off[d][pairs[p][0]] = a ? -1 : +1;
                off[d][pairs[p][1]] = b ? -1 : +1;
            }
}

template <typename R> void build_squared_coarse(dwf_ctx *c, Level &L, Level &Lc, const C<R> *Q, C<R> *W) {
    DWF_REQUIRE(L.index == 0, DWF_EINVAL, "the squared coarsening starts from the fine lattice");
    // a direction of lattice extent 1 hops back onto the same site: its terms
    // stay in T_0 (block-internal) and its pieces T_sigma are zero
    for (int i = 0; i < 4; ++i)
        DWF_REQUIRE(L.block[i] >= 2 || L.lg.g.L[i] == 1, DWF_EINVAL,
                    "the squared coarse stencil needs block extents >= 2");
    const int nv = L.nv;
    const int64_t nc = Lc.lg.g.V, np = (int64_t)nv * nv;
    dslash(c, W, Q, false, nv);  // W_l = D q_l
    FaceMap m;
    for (int i = 0; i < 4; ++i) {
        m.L[i] = L.lg.g.L[i];
        m.b[i] = L.block[i];
        m.Lc[i] = m.L[i] / m.b[i];
    }
    m.Ls = L.lg.g.Ls;
    m.run = 12;
    m.nelem = L.lg.nelem;
    int64_t nfmax = 0;
    for (int mu = 0; mu < 4; ++mu)
        nfmax = std::max<int64_t>(nfmax, (int64_t)m.b[0] * m.b[1] * m.b[2] * m.b[3] / m.b[mu]);
    const int64_t nfe = nfmax * 12 * m.Ls;
    DevBuf Hf(sizeof(C<R>) * (size_t)(8 * nv * nc * nfe));
    const C<R> *Ul = std::is_same<R, double>::value ? (const C<R> *)c->U64.p : (const C<R> *)c->U32.p;
    face_terms_kernel<R><<<dim3((unsigned)nc, 8, (unsigned)nv), 256, 0, c->stream>>>(Hf.as<C<R>>(), Q, Ul, L.lg.g, m,
                                                                                      nc, nfe);
    DWF_CHECK_LAUNCH();
    for (int dd = 0; dd < 8; ++dd) {
        if (m.L[dd >> 1] == 1) {
            DWF_CUDA(cudaMemsetAsync(Hf.as<C<R>>() + (size_t)dd * nv * nc * nfe, 0,
                                     sizeof(C<R>) * (size_t)nv * nc * nfe, c->stream));
            continue;
        }
        subtract_faces_kernel<R><<<dim3((unsigned)nc, (unsigned)nv), 256, 0, c->stream>>>(W, Hf.as<C<R>>(), m, nc, nfe,
                                                                                          dd);
        DWF_CHECK_LAUNCH();
    }
    DevBuf Gp(sizeof(double2) * (size_t)(nc * SQ_PAIRS * np));
    const PairTable pt = make_pairs();
    const int ch = (int)std::max<int64_t>(1, (46 * 1024) / ((int64_t)2 * nv * sizeof(C<R>)));
    const size_t smem = (size_t)2 * nv * ch * sizeof(C<R>);
    dim3 grid((unsigned)nc, SQ_PAIRS);
#define PK(NV) \
    pair_gram_kernel<NV, R><<<grid, 256, smem, c->stream>>>(Gp.as<double2>(), W, Hf.as<C<R>>(), m, pt, nc, nfe, ch)
    NV_DISPATCH2(nv, PK);
#undef PK
    DWF_CHECK_LAUNCH();
    Lc.npts = 33;
    const size_t yb = sizeof(double2) * (size_t)(nc * 33 * np);
    if (Lc.Y64.bytes < yb) Lc.Y64.alloc(yb);
    const unsigned blocks = (unsigned)std::min<int64_t>((nc * 33 * np + 255) / 256, (int64_t)c->sm_count * 16);
    assemble_squared_kernel<<<blocks, 256, 0, c->stream>>>(Lc.Y64.as<double2>(), Gp.as<double2>(), Lc.lg.g, pt, nv);
    DWF_CHECK_LAUNCH();
    convert_coarse_links(c, Lc);
    // Hf and Gp are freed on return: finish with them first
    DWF_CUDA(cudaStreamSynchronize(c->stream));
}

template void build_squared_coarse<double>(dwf_ctx *, Level &, Level &, const double2 *, double2 *);
template void build_squared_coarse<float>(dwf_ctx *, Level &, Level &, const float2 *, float2 *);

template void build_coarse_from<double>(dwf_ctx *, Level &, Level &, const double2 *, double2 *);
template void build_coarse_from<float>(dwf_ctx *, Level &, Level &, const float2 *, float2 *);

template void coarse_apply<double>(dwf_ctx *, const Level &, double2 *, const double2 *, bool);
template void coarse_apply<float>(dwf_ctx *, const Level &, float2 *, const float2 *, bool);

}  // namespace dwf
