// Block transfer operators (Sec. 1: restrictor R and prolongator P with
// R P = 1_c; Sec. 2: near-null vectors cut into blocks, the blocks cover the
// whole fifth dimension).
//
// A coarse site owns a block of bx*by*bz*bt sites of the finer level with all
// their components and all s.  In the s-fastest layout the elements of one
// finer site are contiguous (ncomp*Ls of them), so a CTA that walks the
// block site by site reads whole contiguous runs.  One CTA per coarse site;
// reductions over the block use warp shuffles, then shared memory.
#include "mg.cuh"

namespace dwf {

namespace {

struct BlockMap {
    int L[4];        // finer lattice
    int b[4];        // block
    int Lc[4];       // coarse lattice
    int run;         // contiguous elements per finer site = ncomp * Ls
    int64_t bsites;  // sites per block
    int64_t nelem;   // elements per finer field
};

__device__ __forceinline__ int64_t block_elem_addr(const BlockMap &m, int64_t xc, int64_t e) {
    int64_t i = e / m.run;
    int rem = (int)(e - i * m.run);
    int c[4], o[4];
    int64_t t = xc;
    c[0] = (int)(t % m.Lc[0]); t /= m.Lc[0];
    c[1] = (int)(t % m.Lc[1]); t /= m.Lc[1];
    c[2] = (int)(t % m.Lc[2]); c[3] = (int)(t / m.Lc[2]);
    o[0] = (int)(i % m.b[0]); i /= m.b[0];
    o[1] = (int)(i % m.b[1]); i /= m.b[1];
    o[2] = (int)(i % m.b[2]); o[3] = (int)(i / m.b[2]);
    int64_t site = (((int64_t)(c[3] * m.b[3] + o[3]) * m.L[2] + (c[2] * m.b[2] + o[2])) * m.L[1] +
                    (c[1] * m.b[1] + o[1])) * m.L[0] + (c[0] * m.b[0] + o[0]);
    return site * m.run + rem;
}

// element address of the first element of the i-th finer site of block xc
__device__ __forceinline__ int64_t block_site_addr(const BlockMap &m, int64_t xc, int64_t i) {
    int c[4], o[4];
    int64_t t = xc;
    c[0] = (int)(t % m.Lc[0]); t /= m.Lc[0];
    c[1] = (int)(t % m.Lc[1]); t /= m.Lc[1];
    c[2] = (int)(t % m.Lc[2]); c[3] = (int)(t / m.Lc[2]);
    o[0] = (int)(i % m.b[0]); i /= m.b[0];
    o[1] = (int)(i % m.b[1]); i /= m.b[1];
    o[2] = (int)(i % m.b[2]); o[3] = (int)(i / m.b[2]);
    int64_t site = (((int64_t)(c[3] * m.b[3] + o[3]) * m.L[2] + (c[2] * m.b[2] + o[2])) * m.L[1] +
                    (c[1] * m.b[1] + o[1])) * m.L[0] + (c[0] * m.b[0] + o[0]);
    return site * m.run;
}

BlockMap make_map(const Level &L) {
    BlockMap m;
    for (int i = 0; i < 4; ++i) {
        m.L[i] = L.lg.g.L[i];
        m.b[i] = L.block[i];
        m.Lc[i] = m.L[i] / m.b[i];
    }
    m.run = L.lg.ncomp * L.lg.g.Ls;
    m.bsites = (int64_t)m.b[0] * m.b[1] * m.b[2] * m.b[3];
    m.nelem = L.lg.nelem;
    return m;
}

int64_t ncoarse(const BlockMap &m) { return (int64_t)m.Lc[0] * m.Lc[1] * m.Lc[2] * m.Lc[3]; }

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
}

constexpr int TT = 256;  // threads per CTA of the block kernels

// basis element in the vector precision; the basis may be stored in FP16
template <typename R, typename QT> struct QLoad;
template <typename R> struct QLoad<R, C<R>> {
    static __device__ __forceinline__ C<R> get(const C<R> *Q, int64_t i) { return Q[i]; }
};
template <> struct QLoad<float, __half2> {
    static __device__ __forceinline__ float2 get(const __half2 *Q, int64_t i) { return __half22float2(Q[i]); }
};

template <typename R, typename QT, int NV>
__global__ void __launch_bounds__(TT) restrict_kernel(C<R> *__restrict__ cout, const C<R> *__restrict__ f,
                                                      const QT *__restrict__ Q, BlockMap m) {
    __shared__ C<R> red[TT / 32][NV];
    const int64_t xc = blockIdx.x;
    const int64_t ne = m.bsites * m.run;
    C<R> acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = mk<R>(0, 0);
    for (int64_t e = threadIdx.x; e < ne; e += TT) {
        int64_t a = block_elem_addr(m, xc, e);
        C<R> v = f[a];
#pragma unroll
        for (int k = 0; k < NV; ++k) cfmac(acc[k], QLoad<R, QT>::get(Q, k * m.nelem + a), v);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        C<R> s = warp_sum(acc[k]);
        if (l == 0) red[w][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        C<R> s = mk<R>(0, 0);
#pragma unroll
        for (int i = 0; i < TT / 32; ++i) s = s + red[i][threadIdx.x];
        cout[xc * NV + threadIdx.x] = s;
    }
}

template <typename R, typename QT, int NV>
__global__ void __launch_bounds__(TT) prolong_kernel(C<R> *__restrict__ f, const C<R> *__restrict__ cin,
                                                     const QT *__restrict__ Q, BlockMap m, int accumulate) {
    __shared__ C<R> cs[NV];
    const int64_t xc = blockIdx.x;
    if (threadIdx.x < NV) cs[threadIdx.x] = cin[xc * NV + threadIdx.x];
    __syncthreads();
    const int64_t ne = m.bsites * m.run;
    for (int64_t e = threadIdx.x; e < ne; e += TT) {
        int64_t a = block_elem_addr(m, xc, e);
        C<R> v = accumulate ? f[a] : mk<R>(0, 0);
#pragma unroll
        for (int k = 0; k < NV; ++k) cfma(v, QLoad<R, QT>::get(Q, k * m.nelem + a), cs[k]);
        f[a] = v;
    }
}

// G[xc][k][l] = sum_{e in block} conj(A_k(e)) B_l(e), FP64 accumulation.
// Chunks of CH elements of all NV fields of A and B are staged in shared
// memory; each thread owns a few (k,l) pairs.
template <typename R, int NV, int CH>
__global__ void __launch_bounds__(TT) gram_kernel(double2 *__restrict__ G, const C<R> *__restrict__ A,
                                                  const C<R> *__restrict__ B, BlockMap m) {
    __shared__ C<R> sA[NV][CH];
    __shared__ C<R> sB[NV][CH];
    constexpr int NP = NV * NV;
    constexpr int PPT = (NP + TT - 1) / TT;
    const int64_t xc = blockIdx.x;
    const int64_t ne = m.bsites * m.run;
    double2 acc[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) acc[q] = make_double2(0, 0);
    for (int64_t e0 = 0; e0 < ne; e0 += CH) {
        for (int j = threadIdx.x; j < NV * CH; j += TT) {
            int k = j / CH, e = j - k * CH;
            C<R> a = mk<R>(0, 0), b = mk<R>(0, 0);
            if (e0 + e < ne) {
                int64_t ad = block_elem_addr(m, xc, e0 + e);
                a = A[k * m.nelem + ad];
                b = B[k * m.nelem + ad];
            }
            sA[k][e] = a;
            sB[k][e] = b;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            int p = threadIdx.x + q * TT;
            if (p < NP) {
                int k = p / NV, l = p - k * NV;
                C<R> s = mk<R>(0, 0);
#pragma unroll 8
                for (int e = 0; e < CH; ++e) cfmac(s, sA[k][e], sB[l][e]);
                acc[q].x += (double)s.x;
                acc[q].y += (double)s.y;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        int p = threadIdx.x + q * TT;
        if (p < NP) G[xc * NP + p] = acc[q];
    }
}

// Cholesky G = R^+ R (R upper triangular, positive diagonal) and Rinv = R^-1,
// one thread per coarse site, in FP64.  info[xc] = 0 or (1 + failing column).
__global__ void chol_inv_kernel(const double2 *__restrict__ G, double2 *__restrict__ Rm,
                                double2 *__restrict__ Ri, int *info, int64_t nc, int nv) {
    int64_t xc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (xc >= nc) return;
    const double2 *g = G + xc * nv * nv;
    double2 *r = Rm + xc * nv * nv;
    double2 *ri = Ri + xc * nv * nv;
    int bad = 0;
    for (int i = 0; i < nv * nv; ++i) { r[i] = make_double2(0, 0); ri[i] = make_double2(0, 0); }
    for (int j = 0; j < nv && !bad; ++j) {
        double d = g[j * nv + j].x;
        for (int i = 0; i < j; ++i) d -= r[i * nv + j].x * r[i * nv + j].x + r[i * nv + j].y * r[i * nv + j].y;
        if (!(d > 1e-28 * fabs(g[j * nv + j].x)) || !(d > 0.0)) { bad = j + 1; break; }
        double rd = sqrt(d);
        r[j * nv + j] = make_double2(rd, 0);
        for (int k = j + 1; k < nv; ++k) {
            double2 s = g[j * nv + k];
            for (int i = 0; i < j; ++i) {
                double2 t = cmulc(r[i * nv + j], r[i * nv + k]);
                s.x -= t.x;
                s.y -= t.y;
            }
            r[j * nv + k] = make_double2(s.x / rd, s.y / rd);
        }
    }
    info[xc] = bad;
    if (bad) return;
    // back substitution: R X = I, X upper triangular
    for (int col = 0; col < nv; ++col) {
        for (int i = col; i >= 0; --i) {
            double2 s = make_double2(i == col ? 1.0 : 0.0, 0.0);
            for (int k = i + 1; k <= col; ++k) {
                double2 t = cmul(r[i * nv + k], ri[k * nv + col]);
                s.x -= t.x;
                s.y -= t.y;
            }
            double dinv = 1.0 / r[i * nv + i].x;
            ri[i * nv + col] = make_double2(s.x * dinv, s.y * dinv);
        }
    }
}

// Q_l <- sum_{k <= l} Q_k Rinv[k][l] in place, per block.
template <typename R, int NV>
__global__ void __launch_bounds__(TT) apply_rinv_kernel(C<R> *__restrict__ Q, const double2 *__restrict__ Ri, BlockMap m) {
    __shared__ C<R> r[NV * NV];
    const int64_t xc = blockIdx.x;
    for (int i = threadIdx.x; i < NV * NV; i += TT) r[i] = cvt<C<R>, double2>(Ri[xc * NV * NV + i]);
    __syncthreads();
    const int64_t ne = m.bsites * m.run;
    for (int64_t e = threadIdx.x; e < ne; e += TT) {
        int64_t a = block_elem_addr(m, xc, e);
        C<R> v[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = Q[k * m.nelem + a];
#pragma unroll
        for (int l = NV - 1; l >= 0; --l) {
            C<R> s = mk<R>(0, 0);
#pragma unroll
            for (int k = 0; k <= l; ++k) cfma(s, v[k], r[k * NV + l]);
            Q[l * m.nelem + a] = s;
        }
    }
}

// Gamma split of adaptive vectors into Q (see mg.cuh).
template <typename R>
__global__ void gamma_split_kernel(C<R> *__restrict__ Q, const double2 *__restrict__ v, int nadapt, int split,
                                   int64_t nelem, int ncomp, int Ls, int fine) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nelem; i += (int64_t)gridDim.x * blockDim.x) {
        int s = (int)(i % Ls);
        int64_t sc = i / Ls;
        int comp = (int)(sc % ncomp);
        int64_t site = sc / ncomp;
        for (int j = 0; j < nadapt; ++j) {
            double2 a = v[j * nelem + i];
            if (!split) {
                Q[j * nelem + i] = cvt<C<R>, double2>(a);
                continue;
            }
            double2 ga;  // (Gamma v)(i)
            if (fine) {
                double2 b = v[j * nelem + (site * ncomp + comp) * Ls + (Ls - 1 - s)];
                double g5 = comp < 6 ? 1.0 : -1.0;
                ga = make_double2(g5 * b.x, g5 * b.y);
            } else {
                double gc = (comp & 1) ? -1.0 : 1.0;
                ga = make_double2(gc * a.x, gc * a.y);
            }
            Q[(2 * j) * nelem + i] = cvt<C<R>, double2>(make_double2(0.5 * (a.x + ga.x), 0.5 * (a.y + ga.y)));
            Q[(2 * j + 1) * nelem + i] = cvt<C<R>, double2>(make_double2(0.5 * (a.x - ga.x), 0.5 * (a.y - ga.y)));
        }
    }
}

#define NV_DISPATCH(nv, MACRO)                                      \
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

}  // namespace

template <typename R, typename QT>
void restrict_q(dwf_ctx *c, const Level &L, C<R> *cout, const C<R> *fin, const QT *Q) {
    BlockMap m = make_map(L);
    ProfScope ps(c, K_RESTRICT);
#define RK(NV) restrict_kernel<R, QT, NV><<<(unsigned)ncoarse(m), TT, 0, c->stream>>>(cout, fin, Q, m)
    NV_DISPATCH(L.nv, RK);
#undef RK
    DWF_CHECK_LAUNCH();
}

template <typename R, typename QT>
void prolong_q(dwf_ctx *c, const Level &L, C<R> *fout, const C<R> *cin, const QT *Q, bool acc) {
    BlockMap m = make_map(L);
    ProfScope ps(c, K_PROLONG);
#define PK(NV) prolong_kernel<R, QT, NV><<<(unsigned)ncoarse(m), TT, 0, c->stream>>>(fout, cin, Q, m, acc ? 1 : 0)
    NV_DISPATCH(L.nv, PK);
#undef PK
    DWF_CHECK_LAUNCH();
}

template <typename R> void restrict_(dwf_ctx *c, const Level &L, C<R> *cout, const C<R> *fin, const C<R> *Q) {
    restrict_q<R, C<R>>(c, L, cout, fin, Q);
}
template <typename R> void prolong_(dwf_ctx *c, const Level &L, C<R> *fout, const C<R> *cin, const C<R> *Q, bool acc) {
    prolong_q<R, C<R>>(c, L, fout, cin, Q, acc);
}
void restrict_h(dwf_ctx *c, const Level &L, float2 *cout, const float2 *fin, const __half2 *Q) {
    restrict_q<float, __half2>(c, L, cout, fin, Q);
}
void prolong_h(dwf_ctx *c, const Level &L, float2 *fout, const float2 *cin, const __half2 *Q, bool acc) {
    prolong_q<float, __half2>(c, L, fout, cin, Q, acc);
}

namespace {
// Batched restriction: c_r(xc, k) = sum_e conj(Q_k(e)) f_r(e) for NB right-
// hand sides r0 .. r0+NB-1 (masked beyond nrhs), one CTA per coarse site.
// Warp w owns basis rows k = w*KG .. w*KG+KG-1 and all NB right-hand sides
// (KG*NB accumulators per lane); lanes stream over the block's elements, so
// every basis value is read once and each field value is read by the 8
// warps of the CTA (L1).  Lane partial sums are reduced with shuffles.
// CTA b handles coarse site b / ngroups and the right-hand sides
// r0 = (b % ngroups) * NB ...: the CTAs of one coarse site are adjacent, so
// its basis block is read from HBM once and from L2 by the others.
template <typename R, int NV, int NB>
__global__ void __launch_bounds__(TT, 4) restrict_b_kernel(C<R> *__restrict__ cout, const C<R> *__restrict__ f,
                                                        const C<R> *__restrict__ Q, BlockMap m, int nrhs, int ngroups,
                                                        int64_t cstride) {
    constexpr int NW = TT / 32;
    constexpr int KG = (NV + NW - 1) / NW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k0 = warp * KG;
    const int64_t xc = blockIdx.x / ngroups;
    const int r0 = (int)(blockIdx.x - xc * ngroups) * NB;
    C<R> acc[KG][NB];
#pragma unroll
    for (int a = 0; a < KG; ++a)
#pragma unroll
        for (int r = 0; r < NB; ++r) acc[a][r] = mk<R>(0, 0);
    const int nrb = nrhs - r0 < NB ? nrhs - r0 : NB;
    // walk the block site by site (one address computation per site); the
    // lanes stream over the site's contiguous run of components x s
    for (int64_t i = 0; i < m.bsites; ++i) {
        const int64_t sa = block_site_addr(m, xc, i);
#pragma unroll 1
        for (int j = lane; j < m.run; j += 32) {
            const int64_t ad = sa + j;
            C<R> fv[NB];
#pragma unroll
            for (int r = 0; r < NB; ++r) fv[r] = r < nrb ? f[(int64_t)(r0 + r) * m.nelem + ad] : mk<R>(0, 0);
#pragma unroll
            for (int a = 0; a < KG; ++a) {
                if (k0 + a < NV) {
                    const C<R> q = Q[(k0 + a) * m.nelem + ad];
#pragma unroll
                    for (int r = 0; r < NB; ++r) cfmac(acc[a][r], q, fv[r]);
                }
            }
        }
    }
#pragma unroll
    for (int a = 0; a < KG; ++a)
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            C<R> v = acc[a][r];
            for (int o = 16; o > 0; o >>= 1) {
                v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
            }
            if (lane == 0 && k0 + a < NV && r < nrb) cout[(int64_t)(r0 + r) * cstride + xc * NV + k0 + a] = v;
        }
}

// Batched prolongation: f_r(e) (+)= sum_k Q_k(e) c_r(xc, k) for all nrhs
// right-hand sides; each basis value is loaded once for all of them.
template <typename R, int NV>
__global__ void __launch_bounds__(TT) prolong_b_kernel(C<R> *__restrict__ f, const C<R> *__restrict__ cin,
                                                       const C<R> *__restrict__ Q, BlockMap m, int nrhs,
                                                       int64_t cstride, int accumulate) {
    extern __shared__ unsigned char cs_raw[];
    C<R> *cs = reinterpret_cast<C<R> *>(cs_raw);  // [nrhs][NV]
    const int64_t xc = blockIdx.x;
    for (int i = threadIdx.x; i < nrhs * NV; i += TT) cs[i] = cin[(int64_t)(i / NV) * cstride + xc * NV + i % NV];
    __syncthreads();
    const int64_t ne = m.bsites * m.run;
    for (int64_t e = threadIdx.x; e < ne; e += TT) {
        const int64_t a = block_elem_addr(m, xc, e);
        C<R> q[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) q[k] = Q[k * m.nelem + a];
        for (int r = 0; r < nrhs; ++r) {
            C<R> v = accumulate ? f[(int64_t)r * m.nelem + a] : mk<R>(0, 0);
#pragma unroll
            for (int k = 0; k < NV; ++k) cfma(v, q[k], cs[r * NV + k]);
            f[(int64_t)r * m.nelem + a] = v;
        }
    }
}

__global__ void to_half_kernel(__half2 *__restrict__ out, const float2 *__restrict__ in, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __floats2half2_rn(in[i].x, in[i].y);
}
}  // namespace

template <typename R>
void restrict_batch(dwf_ctx *c, const Level &L, C<R> *cout, const C<R> *fin, const C<R> *Q, int nrhs) {
    BlockMap m = make_map(L);
    ProfScope ps(c, K_RESTRICT, nrhs);
    const int64_t cstride = ncoarse(m) * L.nv;
    constexpr int NB = 4;  // right-hand sides per CTA
    const int ngroups = (nrhs + NB - 1) / NB;
    const int64_t nblk = ncoarse(m) * ngroups;
    DWF_REQUIRE(nblk < ((int64_t)1 << 31), DWF_EINVAL, "batched restriction grid too large");
#define RB(NV) restrict_b_kernel<R, NV, NB><<<(unsigned)nblk, TT, 0, c->stream>>>(cout, fin, Q, m, nrhs, ngroups, cstride)
    NV_DISPATCH(L.nv, RB);
#undef RB
    DWF_CHECK_LAUNCH();
}

template <typename R>
void prolong_batch(dwf_ctx *c, const Level &L, C<R> *fout, const C<R> *cin, const C<R> *Q, int nrhs, bool acc) {
    BlockMap m = make_map(L);
    ProfScope ps(c, K_PROLONG, nrhs);
    const int64_t cstride = ncoarse(m) * L.nv;
    const size_t smem = sizeof(C<R>) * (size_t)nrhs * L.nv;
    DWF_REQUIRE(smem <= 46 * 1024, DWF_EINVAL, "too many right-hand sides for the batched prolongation");
#define PB(NV) prolong_b_kernel<R, NV><<<(unsigned)ncoarse(m), TT, smem, c->stream>>>(fout, cin, Q, m, nrhs, cstride, acc ? 1 : 0)
    NV_DISPATCH(L.nv, PB);
#undef PB
    DWF_CHECK_LAUNCH();
}

template void restrict_batch<float>(dwf_ctx *, const Level &, float2 *, const float2 *, const float2 *, int);
template void restrict_batch<double>(dwf_ctx *, const Level &, double2 *, const double2 *, const double2 *, int);
template void prolong_batch<float>(dwf_ctx *, const Level &, float2 *, const float2 *, const float2 *, int, bool);
template void prolong_batch<double>(dwf_ctx *, const Level &, double2 *, const double2 *, const double2 *, int, bool);

void basis_to_half(dwf_ctx *c, __half2 *out, const float2 *in, int64_t n) {
    unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 16);
    to_half_kernel<<<blocks, 256, 0, c->stream>>>(out, in, n);
    DWF_CHECK_LAUNCH();
}

template <typename R> void block_gram(dwf_ctx *c, const Level &L, double2 *G, const C<R> *A, const C<R> *B) {
    BlockMap m = make_map(L);
#define GK(NV) gram_kernel<R, NV, (NV > 16 ? 16 : 32)><<<(unsigned)ncoarse(m), TT, 0, c->stream>>>(G, A, B, m)
    NV_DISPATCH(L.nv, GK);
#undef GK
    DWF_CHECK_LAUNCH();
}

template <typename R> bool block_orthonormalise(dwf_ctx *c, Level &L, C<R> *Q) {
    BlockMap m = make_map(L);
    int64_t nc = ncoarse(m);
    size_t gb = sizeof(double2) * nc * L.nv * L.nv;
    if (L.G.bytes < gb) L.G.alloc(gb);
    if (L.F.bytes < gb) L.F.alloc(gb);
    if (L.Rinv.bytes < gb) L.Rinv.alloc(gb);
    if (L.info.bytes < sizeof(int) * nc) L.info.alloc(sizeof(int) * nc);
    std::vector<int> info(nc);
    for (int pass = 0; pass < 2; ++pass) {  // CholQR2
        block_gram<R>(c, L, L.G.as<double2>(), Q, Q);
        chol_inv_kernel<<<(unsigned)((nc + 63) / 64), 64, 0, c->stream>>>(L.G.as<double2>(), L.F.as<double2>(),
                                                                          L.Rinv.as<double2>(), L.info.as<int>(), nc, L.nv);
        DWF_CHECK_LAUNCH();
        DWF_CUDA(cudaMemcpyAsync(info.data(), L.info.p, sizeof(int) * nc, cudaMemcpyDeviceToHost, c->stream));
        DWF_CUDA(cudaStreamSynchronize(c->stream));
        for (int64_t i = 0; i < nc; ++i)
            if (info[i]) return false;
#define AK(NV) apply_rinv_kernel<R, NV><<<(unsigned)nc, TT, 0, c->stream>>>(Q, L.Rinv.as<double2>(), m)
        NV_DISPATCH(L.nv, AK);
#undef AK
        DWF_CHECK_LAUNCH();
    }
    return true;
}

template <typename R> void gamma_split(dwf_ctx *c, const Level &L, C<R> *Q, const double2 *v, int nadapt, bool split) {
    int64_t n = L.lg.nelem;
    unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 16);
    gamma_split_kernel<R><<<blocks, 256, 0, c->stream>>>(Q, v, nadapt, split ? 1 : 0, n, L.lg.ncomp, L.lg.g.Ls,
                                                         L.index == 0 ? 1 : 0);
    DWF_CHECK_LAUNCH();
}

template void restrict_<double>(dwf_ctx *, const Level &, double2 *, const double2 *, const double2 *);
template void restrict_<float>(dwf_ctx *, const Level &, float2 *, const float2 *, const float2 *);
template void prolong_<double>(dwf_ctx *, const Level &, double2 *, const double2 *, const double2 *, bool);
template void prolong_<float>(dwf_ctx *, const Level &, float2 *, const float2 *, const float2 *, bool);
template void block_gram<double>(dwf_ctx *, const Level &, double2 *, const double2 *, const double2 *);
template void block_gram<float>(dwf_ctx *, const Level &, double2 *, const float2 *, const float2 *);
template bool block_orthonormalise<double>(dwf_ctx *, Level &, double2 *);
template bool block_orthonormalise<float>(dwf_ctx *, Level &, float2 *);
template void gamma_split<double>(dwf_ctx *, const Level &, double2 *, const double2 *, int, bool);
template void gamma_split<float>(dwf_ctx *, const Level &, float2 *, const double2 *, int, bool);

}  // namespace dwf
