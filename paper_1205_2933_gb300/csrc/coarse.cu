// The Galerkin coarse operator R A P (Sec. 2, third step of the V-cycle:
// S2 acts on R A P) as a 9-point stencil of dense n x n complex blocks:
//   (A_c c)(x) = Y0(x) c(x) + sum_{mu, dir} Y_{mu,dir}(x) c(x + dir*mu),
// direction index d = 0 (self), 1 + 2*mu (+mu), 2 + 2*mu (-mu); storage
// Y[x][d][k][l].  One fine hop crosses at most one block face, so the
// unsquared operator coarsens to nearest neighbours (Sec. 4 contrasts this
// with the squared operator's 17-site coarse stencil).
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

template <typename R, typename LT, int NV, bool DAG>
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
    for (int d = 0; d < 9; ++d) {
        int64_t other = site;
        // table entry 2 mu: +mu, 2 mu + 1: -mu; D^+ reads the opposite neighbour
        if (d > 0) other = nbr[site * 8 + (DAG ? ((d - 1) ^ 1) : (d - 1))];
        const C<R> *xv = x + other * NV;
        if (!DAG) {
            const int64_t row = ((site * 9 + d) * NV + k) * NV;
#pragma unroll 8
            for (int l = 0; l < NV; ++l) cfma(acc, LinkRead<LT>::template get<R>(Y, row + l), xv[l]);
        } else {
            const int64_t base = (other * 9 + d) * NV * NV + k;
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
                int c[4];
                site_coords(g, site, c);
                int cc[4] = {c[0], c[1], c[2], c[3]};
                cc[mu] += dir;
                bool wrap = (cc[mu] == g.L[mu] || cc[mu] < 0);
                if (cc[mu] == g.L[mu]) cc[mu] = 0;
                if (cc[mu] < 0) cc[mu] = g.L[mu] - 1;
                int64_t nb = site_index(g, cc);
                R coef = (mu == 3 && g.ap && wrap) ? R(0.5) : R(-0.5);
                C<R> acc12[12];
                for (int e = 0; e < 12; ++e) acc12[e] = mk<R>(0, 0);
                C<R> lk[9];
                LinkIO<R>::load(U, dir > 0 ? site : nb, mu, lk);
                if (dir > 0) {
                    switch (mu) {
                        case 0: hop<0, false, R>(acc12, ql, nb, m.Ls, s, lk, -1, coef); break;
                        case 1: hop<1, false, R>(acc12, ql, nb, m.Ls, s, lk, -1, coef); break;
                        case 2: hop<2, false, R>(acc12, ql, nb, m.Ls, s, lk, -1, coef); break;
                        default: hop<3, false, R>(acc12, ql, nb, m.Ls, s, lk, -1, coef); break;
                    }
                } else {
                    switch (mu) {
                        case 0: hop<0, true, R>(acc12, ql, nb, m.Ls, s, lk, +1, coef); break;
                        case 1: hop<1, true, R>(acc12, ql, nb, m.Ls, s, lk, +1, coef); break;
                        case 2: hop<2, true, R>(acc12, ql, nb, m.Ls, s, lk, +1, coef); break;
                        default: hop<3, true, R>(acc12, ql, nb, m.Ls, s, lk, +1, coef); break;
                    }
                }
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
    if (dag) coarse_apply_kernel<R, LT, NV, true><<<grid, 256, 0, c->stream>>>(y, x, Y, g, nbrt);            \
    else coarse_apply_kernel<R, LT, NV, false><<<grid, 256, 0, c->stream>>>(y, x, Y, g, nbrt)
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
    int64_t n = L.lg.g.V * 9 * (int64_t)L.lg.ncomp * L.lg.ncomp;
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

template void build_coarse_from<double>(dwf_ctx *, Level &, Level &, const double2 *, double2 *);
template void build_coarse_from<float>(dwf_ctx *, Level &, Level &, const float2 *, float2 *);

template void coarse_apply<double>(dwf_ctx *, const Level &, double2 *, const double2 *, bool);
template void coarse_apply<float>(dwf_ctx *, const Level &, float2 *, const float2 *, bool);

}  // namespace dwf
