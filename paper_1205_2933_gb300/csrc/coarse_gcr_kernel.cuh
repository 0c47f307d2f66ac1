// Kernel of the fused coarsest-level GCR (one cooperative launch), shared by
// the 9-point (R D P) and 33-point (P^+ D^+ D P) stencils; each includer
// instantiates one stencil size.
#pragma once

#include <cooperative_groups.h>

#include "mg.cuh"

namespace dwf {

namespace cg = cooperative_groups;

namespace {

constexpr int CT = 256;        // threads per CTA
constexpr int MAXR = 32;       // maximum restart length of the fused solver

template <typename LT> struct LRead;
template <> struct LRead<double2> {
    template <typename R> static __device__ __forceinline__ C<R> get(const double2 *Y, int64_t i) { return cvt<C<R>, double2>(Y[i]); }
};
template <> struct LRead<float2> {
    template <typename R> static __device__ __forceinline__ C<R> get(const float2 *Y, int64_t i) { return cvt<C<R>, float2>(Y[i]); }
};
template <> struct LRead<__nv_bfloat162> {
    template <typename R> static __device__ __forceinline__ C<R> get(const __nv_bfloat162 *Y, int64_t i) {
        return cvt<C<R>, float2>(__bfloat1622float2(Y[i]));
    }
};
template <> struct LRead<__half2> {
    template <typename R> static __device__ __forceinline__ C<R> get(const __half2 *Y, int64_t i) {
        return cvt<C<R>, float2>(__half22float2(Y[i]));
    }
};

template <typename R, typename LT> struct Args {
    const LT *Y;
    const int *nbr;    // neighbour table [V][NPTS - 1]
    Geom g;            // coarse lattice (g.V sites)
    const C<R> *b;
    C<R> *x, *r, *Z, *W;   // Z, W: restart vectors each
    double2 *part;     // [3][MAXR + 2][gridDim.x] FP64 partial sums
    double tol;
    int maxiter, restart;
    int *iters;        // accumulates the iteration count
};

// out = A in on the owned sites [s0, s1): one warp per site, lane l holds
// column l of every link row (coalesced loads) and the 9 neighbour values
// in[nbr_d][l]; each output row is a warp-wide sum over l.
template <typename R, typename LT, int NV, int NPTS>
__device__ void apply_owned(const Args<R, LT> &a, C<R> *out, const C<R> *in, int64_t s0, int64_t s1) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool on = lane < NV;
    for (int64_t site = s0 + warp; site < s1; site += CT / 32) {
        C<R> xv[NPTS];
#pragma unroll
        for (int d = 0; d < NPTS; ++d) {
            const int o = d > 0 ? a.nbr[site * (NPTS - 1) + d - 1] : (int)site;
            xv[d] = on ? in[o * NV + lane] : mk<R>(0, 0);
        }
        const LT *Ys = a.Y + site * NPTS * NV * NV;
        // unrolled so that the link loads of several row pairs are in flight
        // together (the loop is bound by L2 latency, not bandwidth)
#pragma unroll 4
        for (int k = 0; k < NV; k += 2) {
            R r0 = 0, i0 = 0, r1 = 0, i1 = 0;
            if (on) {
#pragma unroll
                for (int d = 0; d < NPTS; ++d) {
                    C<R> y0 = LRead<LT>::template get<R>(Ys, ((int64_t)d * NV + k) * NV + lane);
                    C<R> y1 = LRead<LT>::template get<R>(Ys, ((int64_t)d * NV + k + 1) * NV + lane);
                    r0 += y0.x * xv[d].x - y0.y * xv[d].y;
                    i0 += y0.x * xv[d].y + y0.y * xv[d].x;
                    r1 += y1.x * xv[d].x - y1.y * xv[d].y;
                    i1 += y1.x * xv[d].y + y1.y * xv[d].x;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                r0 += __shfl_xor_sync(0xffffffffu, r0, o);
                i0 += __shfl_xor_sync(0xffffffffu, i0, o);
                r1 += __shfl_xor_sync(0xffffffffu, r1, o);
                i1 += __shfl_xor_sync(0xffffffffu, i1, o);
            }
            if (lane == 0) {
                out[site * NV + k] = mk<R>(r0, i0);
                out[site * NV + k + 1] = mk<R>(r1, i1);
            }
        }
    }
    // rows were written by lane 0 of each warp; the element loops that follow
    // read them from other threads of the CTA
    __syncthreads();
}

// Sum over CTAs of part[slot][i][*] for i < k into tot[i] (shared), same
// order in every CTA.  16 lanes per value.
__device__ void gather_totals(const double2 *part, int k, int nb, double2 *tot) {
    for (int i0 = 0; i0 < k; i0 += CT / 16) {
        const int i = i0 + threadIdx.x / 16, lane = threadIdx.x & 15;
        double2 s = make_double2(0, 0);
        if (i < k)
            for (int b = lane; b < nb; b += 16) {
                const volatile double *p = reinterpret_cast<const volatile double *>(part + (size_t)i * nb + b);
                s.x += p[0];
                s.y += p[1];
            }
        for (int o = 8; o > 0; o >>= 1) {
            s.x += __shfl_down_sync(0xffffffffu, s.x, o, 16);
            s.y += __shfl_down_sync(0xffffffffu, s.y, o, 16);
        }
        if (i < k && lane == 0) tot[i] = s;
    }
    __syncthreads();
}

template <typename R, typename LT, int NV, int NPTS>
__global__ void __launch_bounds__(CT) coarse_gcr_kernel(Args<R, LT> a) {
    cg::grid_group grid = cg::this_grid();
    __shared__ double2 red[CT / 32][MAXR + 2];
    __shared__ double2 tot[MAXR + 2];
    const int nb = gridDim.x;
    const int64_t N = a.g.V * NV;
    const int64_t sites = (a.g.V + nb - 1) / nb;   // whole sites per CTA
    const int64_t s0 = blockIdx.x * sites;
    const int64_t s1 = s0 + sites < a.g.V ? s0 + sites : a.g.V;
    const int64_t e0 = s0 * NV;
    const int64_t e1 = s1 > s0 ? s1 * NV : e0;
    const size_t ps = (size_t)(MAXR + 2) * nb;   // size of one partial-sum region
    double2 *P[3] = {a.part, a.part + ps, a.part + 2 * ps};

    // reduce k complex values per thread into tot[0..k): warp shuffles for
    // all k values, one shared-memory pass across warps, one partial per CTA
    auto reduce = [&](double2 *vals, int k, double2 *Pr) {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int i = 0; i < k; ++i) {
            double2 t = vals[i];
            for (int o = 16; o > 0; o >>= 1) {
                t.x += __shfl_down_sync(0xffffffffu, t.x, o);
                t.y += __shfl_down_sync(0xffffffffu, t.y, o);
            }
            if (lane == 0) red[w][i] = t;
        }
        __syncthreads();
        if (threadIdx.x < k) {
            double2 t = make_double2(0, 0);
            for (int j = 0; j < CT / 32; ++j) {
                t.x += red[j][threadIdx.x].x;
                t.y += red[j][threadIdx.x].y;
            }
            Pr[(size_t)threadIdx.x * nb + blockIdx.x] = t;
        }
        __threadfence();
        grid.sync();
        gather_totals(Pr, k, nb, tot);
    };

    // x = 0, r = b, |b|^2
    double2 v[MAXR + 2];
    v[0] = make_double2(0, 0);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += CT) {
        a.x[e] = mk<R>(0, 0);
        C<R> bv = a.b[e];
        a.r[e] = bv;
        v[0].x += (double)bv.x * bv.x + (double)bv.y * bv.y;
    }
    reduce(v, 1, P[2]);
    const double bn2 = tot[0].x;
    double rn2 = bn2;
    int it = 0, k = 0;
    if (bn2 > 0.0) {
        const double stop = a.tol * a.tol * bn2;
        while (it < a.maxiter && rn2 > stop) {
            C<R> *Zk = a.Z + (size_t)k * N, *Wk = a.W + (size_t)k * N;
            for (int64_t e = e0 + threadIdx.x; e < e1; e += CT) Zk[e] = a.r[e];
            __threadfence();
            grid.sync();
            apply_owned<R, LT, NV, NPTS>(a, Wk, Zk, s0, s1);
            for (int pass = 0; pass < 2 && k > 0; ++pass) {
                for (int i = 0; i < k; ++i) v[i] = make_double2(0, 0);
                for (int64_t e = e0 + threadIdx.x; e < e1; e += CT) {
                    C<R> w = Wk[e];
                    // loads issued eight at a time before the products (the loop is latency-bound)
                    for (int i0 = 0; i0 < k; i0 += 8) {
                        C<R> u[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (i0 + j < k) u[j] = a.W[(size_t)(i0 + j) * N + e];
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (i0 + j < k) {
                                v[i0 + j].x += (double)u[j].x * w.x + (double)u[j].y * w.y;
                                v[i0 + j].y += (double)u[j].x * w.y - (double)u[j].y * w.x;
                            }
                    }
                }
                reduce(v, k, P[pass]);
                for (int64_t e = e0 + threadIdx.x; e < e1; e += CT) {
                    C<R> w = Wk[e], z = Zk[e];
                    for (int i0 = 0; i0 < k; i0 += 8) {
                        C<R> wi[8], zi[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (i0 + j < k) {
                                wi[j] = a.W[(size_t)(i0 + j) * N + e];
                                zi[j] = a.Z[(size_t)(i0 + j) * N + e];
                            }
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (i0 + j < k) {
                                const R br = (R)tot[i0 + j].x, bi = (R)tot[i0 + j].y;
                                w.x -= br * wi[j].x - bi * wi[j].y;
                                w.y -= br * wi[j].y + bi * wi[j].x;
                                z.x -= br * zi[j].x - bi * zi[j].y;
                                z.y -= br * zi[j].y + bi * zi[j].x;
                            }
                    }
                    Wk[e] = w;
                    Zk[e] = z;
                }
                __syncthreads();  // tot is rewritten by the next reduction
            }
            v[0] = v[1] = make_double2(0, 0);
            for (int64_t e = e0 + threadIdx.x; e < e1; e += CT) {
                C<R> w = Wk[e], rr = a.r[e];
                v[0].x += (double)w.x * w.x + (double)w.y * w.y;
                v[1].x += (double)w.x * rr.x + (double)w.y * rr.y;
                v[1].y += (double)w.x * rr.y - (double)w.y * rr.x;
            }
            reduce(v, 2, P[2]);
            const double ww = tot[0].x;
            if (!(ww > 0.0)) break;  // breakdown: same decision in every CTA
            const double inv = 1.0 / sqrt(ww);
            const double ar = tot[1].x * inv, ai = tot[1].y * inv;
            const R sc = (R)inv, arr = (R)ar, aii = (R)ai;
            for (int64_t e = e0 + threadIdx.x; e < e1; e += CT) {
                C<R> z = Zk[e], w = Wk[e], xx = a.x[e], rr = a.r[e];
                z.x *= sc; z.y *= sc; w.x *= sc; w.y *= sc;
                xx.x += arr * z.x - aii * z.y;
                xx.y += arr * z.y + aii * z.x;
                rr.x -= arr * w.x - aii * w.y;
                rr.y -= arr * w.y + aii * w.x;
                Zk[e] = z; Wk[e] = w; a.x[e] = xx; a.r[e] = rr;
            }
            rn2 -= ar * ar + ai * ai;
            ++it;
            ++k;
            __syncthreads();
            if (k == a.restart || rn2 <= stop) {
                // true residual r = b - A x
                __threadfence();
                grid.sync();
                apply_owned<R, LT, NV, NPTS>(a, a.r, a.x, s0, s1);
                v[0] = make_double2(0, 0);
                for (int64_t e = e0 + threadIdx.x; e < e1; e += CT) {
                    C<R> bv = a.b[e], ax = a.r[e];
                    C<R> rr = mk<R>(bv.x - ax.x, bv.y - ax.y);
                    a.r[e] = rr;
                    v[0].x += (double)rr.x * rr.x + (double)rr.y * rr.y;
                }
                reduce(v, 1, P[2]);
                rn2 = tot[0].x;
                k = 0;
                __syncthreads();
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.iters, it);
}

// Launch the solver for a stencil of NPTS points (9: R D P; 33: the squared
// operator's P^+ D^+ D P).
template <typename R, typename LT, int NPTS>
void launch_t(dwf_ctx *c, const Level &L, const LT *Y, C<R> *x, const C<R> *b, C<R> *r, C<R> *Z, C<R> *W,
                     double2 *part, int *iters, double tol, int maxiter, int restart) {
    Args<R, LT> a;
    a.Y = Y;
    a.nbr = L.nbr.as<int>();
    a.g = L.lg.g;
    a.b = b;
    a.x = x;
    a.r = r;
    a.Z = Z;
    a.W = W;
    a.part = part;
    a.tol = tol;
    a.maxiter = maxiter;
    a.restart = restart;
    a.iters = iters;
    void *kargs[] = {&a};
    const int n = L.lg.ncomp;
    const int64_t N = L.lg.g.V * n;
    int64_t nblk = (N + CT - 1) / CT;
    if (nblk > c->sm_count) nblk = c->sm_count;
    if (nblk < 1) nblk = 1;
    dim3 grid((unsigned)nblk), block(CT);
    void *fn = nullptr;
    switch (n) {
        case 2: fn = (void *)coarse_gcr_kernel<R, LT, 2, NPTS>; break;
        case 4: fn = (void *)coarse_gcr_kernel<R, LT, 4, NPTS>; break;
        case 6: fn = (void *)coarse_gcr_kernel<R, LT, 6, NPTS>; break;
        case 8: fn = (void *)coarse_gcr_kernel<R, LT, 8, NPTS>; break;
        case 12: fn = (void *)coarse_gcr_kernel<R, LT, 12, NPTS>; break;
        case 16: fn = (void *)coarse_gcr_kernel<R, LT, 16, NPTS>; break;
        case 24: fn = (void *)coarse_gcr_kernel<R, LT, 24, NPTS>; break;
        case 32: fn = (void *)coarse_gcr_kernel<R, LT, 32, NPTS>; break;
        default: throw Error{DWF_EINVAL, "unsupported Nvec"};
    }
    int per_sm = 0;
    DWF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, CT, 0));
    DWF_REQUIRE(per_sm >= 1, DWF_ECUDA, "fused coarse solver cannot be co-resident");
    DWF_CUDA(coop_launch(c, fn, grid, block, kargs, 0));
    DWF_CHECK_LAUNCH();
}

}  // namespace

}  // namespace dwf
