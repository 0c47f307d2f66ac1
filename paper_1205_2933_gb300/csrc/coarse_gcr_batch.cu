// The coarsest-level solve S2 of the V-cycle (Sec. 2) for a batch of right-
// hand sides as one cooperative kernel: restarted GCR on the 9-point coarse
// stencil, all right-hand sides in lockstep through the same grid barriers.
//
// Same algorithm per right-hand side as the one-RHS fused solver
// (coarse_gcr.cu): classical Gram-Schmidt twice against the stored
// directions, |w| normalisation, x += <w,r> z, r -= <w,r> w, true residual
// at each restart.  A right-hand side leaves the lockstep when its residual
// estimate meets the tolerance or its iterations reach the limit.  The grid
// owns contiguous site slices of every vector; a reduction writes one FP64
// partial per CTA and value, CTA j then adds the partials of values j,
// j + grid, ... in a fixed order, and after a second barrier every CTA reads
// the same totals, so all CTAs take identical decisions.
#include <cooperative_groups.h>

#include <type_traits>

#include "mg.cuh"

namespace cg = cooperative_groups;

namespace dwf {

namespace {

constexpr int BCT = 256;                      // threads per CTA
constexpr int BMAXR = 16;                     // restart length
constexpr int BMAXB = 16;                     // right-hand sides per launch
constexpr int MAXV = (BMAXR + 2) * BMAXB;     // reduced values per phase

template <typename LT> struct BLRead;
template <> struct BLRead<double2> {
    template <typename R> static __device__ __forceinline__ C<R> get(const double2 *Y, int64_t i) { return cvt<C<R>, double2>(Y[i]); }
};
template <> struct BLRead<float2> {
    template <typename R> static __device__ __forceinline__ C<R> get(const float2 *Y, int64_t i) { return cvt<C<R>, float2>(Y[i]); }
};
template <> struct BLRead<__nv_bfloat162> {
    template <typename R> static __device__ __forceinline__ C<R> get(const __nv_bfloat162 *Y, int64_t i) {
        return cvt<C<R>, float2>(__bfloat1622float2(Y[i]));
    }
};
template <> struct BLRead<__half2> {
    template <typename R> static __device__ __forceinline__ C<R> get(const __half2 *Y, int64_t i) {
        return cvt<C<R>, float2>(__half22float2(Y[i]));
    }
};

template <typename R, typename LT> struct BArgs {
    const LT *Y;
    const int *nbr;              // neighbour table [V][8]
    Geom g;                      // coarse lattice
    const C<R> *b;               // [nb][N]
    C<R> *x, *r;                 // [nb][N]
    C<R> *Z, *W;                 // [restart][nb][N]
    double2 *part;               // [MAXV][gridDim.x] partial sums
    double2 *tot;                // [MAXV] totals
    double tol;
    int maxiter, restart, nb;
    int *iters;
};

// out_r = A in_r on the owned sites for the active right-hand sides: one warp
// per (site, rhs) task, lane l holds column l; consecutive tasks share the
// site so its links stay in L1.
template <typename R, typename LT, int NV>
__device__ void apply_tasks(const BArgs<R, LT> &a, C<R> *out, const C<R> *in, int N, int s0, int s1,
                            const int *act) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool on = lane < NV;
    const int ntask = (s1 - s0) * a.nb;
    for (int t = warp; t < ntask; t += BCT / 32) {
        const int site = s0 + t / a.nb;
        const int rr = t - (site - s0) * a.nb;
        if (!act[rr]) continue;
        const C<R> *inr = in + rr * N;
        C<R> *outr = out + rr * N;
        C<R> xv[9];
#pragma unroll
        for (int d = 0; d < 9; ++d) {
            const int o = d > 0 ? a.nbr[site * 8 + d - 1] : site;
            xv[d] = on ? inr[o * NV + lane] : mk<R>(0, 0);
        }
        const LT *Ys = a.Y + (int64_t)site * 9 * NV * NV;
#pragma unroll 4
        for (int k = 0; k < NV; k += 2) {
            R r0 = 0, i0 = 0, r1 = 0, i1 = 0;
            if (on) {
#pragma unroll
                for (int d = 0; d < 9; ++d) {
                    C<R> y0 = BLRead<LT>::template get<R>(Ys, (d * NV + k) * NV + lane);
                    C<R> y1 = BLRead<LT>::template get<R>(Ys, (d * NV + k + 1) * NV + lane);
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
                outr[site * NV + k] = mk<R>(r0, i0);
                outr[site * NV + k + 1] = mk<R>(r1, i1);
            }
        }
    }
    __syncthreads();
}

template <typename R, typename LT, int NV>
__global__ void __launch_bounds__(BCT) coarse_gcr_batch_kernel(BArgs<R, LT> a) {
    cg::grid_group grid = cg::this_grid();
    __shared__ double2 red[BCT / 32][MAXV];
    __shared__ double2 tot[MAXV];
    __shared__ double rn2[BMAXB], stop[BMAXB];
    __shared__ int act[BMAXB], its[BMAXB];
    const int nb = a.nb, nblk = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int V = (int)a.g.V, N = V * NV;  // the coarsest field of one RHS is far below 2^31 elements
    const int sites = (V + nblk - 1) / nblk;
    const int s0 = min((int)blockIdx.x * sites, V), s1 = min(s0 + sites, V);
    const int e0 = s0 * NV, e1 = s1 * NV;

    // Element work is spread as items (rr, e): every right-hand side's owned
    // elements padded to whole warps, so the 32 lanes of a warp round share
    // one right-hand side and its partial sums need no segmentation.
    const int E = e1 - e0, Epad = (E + 31) / 32 * 32, nitems = nb * Epad;

    auto zero_red = [&](int nv) {
        for (int q = threadIdx.x; q < (BCT / 32) * nv; q += BCT) red[q / nv][q % nv] = make_double2(0, 0);
        __syncthreads();
    };
    auto wsum = [&](double2 v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, o);
            v.y += __shfl_down_sync(0xffffffffu, v.y, o);
        }
        return v;
    };
    // totals of values 0..nv-1 (summed over warps, then CTAs) into tot[] in every CTA
    auto finish = [&](int nv) {
        __syncthreads();
        for (int p = threadIdx.x; p < nv; p += BCT) {
            double2 s = make_double2(0, 0);
            for (int w = 0; w < BCT / 32; ++w) s = s + red[w][p];
            a.part[(size_t)p * nblk + blockIdx.x] = s;
        }
        __threadfence();
        grid.sync();
        if (warp == 0)
            for (int p = blockIdx.x; p < nv; p += nblk) {
                double2 s = make_double2(0, 0);
                for (int j = lane; j < nblk; j += 32) {
                    const volatile double *q = reinterpret_cast<const volatile double *>(a.part + (size_t)p * nblk + j);
                    s.x += q[0];
                    s.y += q[1];
                }
                s = wsum(s);
                if (lane == 0) a.tot[p] = s;
            }
        __threadfence();
        grid.sync();
        for (int p = threadIdx.x; p < nv; p += BCT) {
            const volatile double *q = reinterpret_cast<const volatile double *>(a.tot + p);
            tot[p] = make_double2(q[0], q[1]);
        }
        __syncthreads();
    };

    // x = 0, r = b, |b|^2 per right-hand side
    zero_red(nb);
    for (int base = warp * 32; base < nitems; base += BCT) {
        const int rr = (int)(base / Epad);
        const int eo = base - rr * Epad + lane;
        double2 v = make_double2(0, 0);
        if (eo < E) {
            const int i = rr * N + e0 + eo;
            a.x[i] = mk<R>(0, 0);
            const C<R> bv = a.b[i];
            a.r[i] = bv;
            v.x = (double)bv.x * bv.x + (double)bv.y * bv.y;
        }
        v = wsum(v);
        if (lane == 0) red[warp][rr] = red[warp][rr] + v;
    }
    finish(nb);
    if (threadIdx.x < nb) {
        const int rr = threadIdx.x;
        rn2[rr] = tot[rr].x;
        stop[rr] = a.tol * a.tol * tot[rr].x;
        act[rr] = (tot[rr].x > 0.0 && a.maxiter > 0) ? 1 : 0;
        its[rr] = 0;
    }
    __syncthreads();
    int k = 0;
    while (true) {
        bool any = false;
        for (int rr = 0; rr < nb; ++rr) any |= act[rr] != 0;
        if (!any) break;
        C<R> *Zk = a.Z + (size_t)k * nb * N, *Wk = a.W + (size_t)k * nb * N;
        for (int base = warp * 32; base < nitems; base += BCT) {
            const int rr = (int)(base / Epad);
            const int eo = base - rr * Epad + lane;
            if (act[rr] && eo < E) Zk[rr * N + e0 + eo] = a.r[rr * N + e0 + eo];
        }
        __threadfence();
        grid.sync();
        apply_tasks<R, LT, NV>(a, Wk, Zk, N, s0, s1, act);
        for (int pass = 0; pass < 2 && k > 0; ++pass) {
            zero_red(k * nb);
            for (int base = warp * 32; base < nitems; base += BCT) {
                const int rr = (int)(base / Epad);
                if (!act[rr]) continue;
                const int eo = base - rr * Epad + lane;
                const bool ok = eo < E;
                const int ie = rr * N + e0 + eo;
                const C<R> w = ok ? Wk[ie] : mk<R>(0, 0);
                C<R> u[BMAXR];
#pragma unroll
                for (int i = 0; i < BMAXR; ++i)
                    if (i < k) u[i] = ok ? a.W[(size_t)i * nb * N + ie] : mk<R>(0, 0);
#pragma unroll
                for (int i = 0; i < BMAXR; ++i)
                    if (i < k) {
                        double2 v = make_double2((double)u[i].x * w.x + (double)u[i].y * w.y,
                                                 (double)u[i].x * w.y - (double)u[i].y * w.x);
                        v = wsum(v);
                        if (lane == 0) red[warp][i * nb + rr] = red[warp][i * nb + rr] + v;
                    }
            }
            finish(k * nb);
            for (int base = warp * 32; base < nitems; base += BCT) {
                const int rr = (int)(base / Epad);
                const int eo = base - rr * Epad + lane;
                if (!act[rr] || eo >= E) continue;
                const int ie = rr * N + e0 + eo;
                C<R> w = Wk[ie], z = Zk[ie];
                C<R> wi[BMAXR], zi[BMAXR];
#pragma unroll
                for (int i = 0; i < BMAXR; ++i)
                    if (i < k) {
                        wi[i] = a.W[(size_t)i * nb * N + ie];
                        zi[i] = a.Z[(size_t)i * nb * N + ie];
                    }
#pragma unroll
                for (int i = 0; i < BMAXR; ++i)
                    if (i < k) {
                        const R br = (R)tot[i * nb + rr].x, bi = (R)tot[i * nb + rr].y;
                        w.x -= br * wi[i].x - bi * wi[i].y;
                        w.y -= br * wi[i].y + bi * wi[i].x;
                        z.x -= br * zi[i].x - bi * zi[i].y;
                        z.y -= br * zi[i].y + bi * zi[i].x;
                    }
                Wk[ie] = w;
                Zk[ie] = z;
            }
            __syncthreads();
        }
        // |w|^2 and <w, r>
        zero_red(2 * nb);
        for (int base = warp * 32; base < nitems; base += BCT) {
            const int rr = (int)(base / Epad);
            if (!act[rr]) continue;
            const int eo = base - rr * Epad + lane;
            double2 v0 = make_double2(0, 0), v1 = make_double2(0, 0);
            if (eo < E) {
                const int ie = rr * N + e0 + eo;
                const C<R> w = Wk[ie], q = a.r[ie];
                v0.x = (double)w.x * w.x + (double)w.y * w.y;
                v1.x = (double)w.x * q.x + (double)w.y * q.y;
                v1.y = (double)w.x * q.y - (double)w.y * q.x;
            }
            v0 = wsum(v0);
            v1 = wsum(v1);
            if (lane == 0) {
                red[warp][rr] = red[warp][rr] + v0;
                red[warp][nb + rr] = red[warp][nb + rr] + v1;
            }
        }
        finish(2 * nb);
        for (int base = warp * 32; base < nitems; base += BCT) {
            const int rr = (int)(base / Epad);
            const int eo = base - rr * Epad + lane;
            if (!act[rr] || eo >= E) continue;
            const double ww = tot[rr].x;
            if (!(ww > 0.0)) continue;  // breakdown: handled below, same in every CTA
            const double inv = 1.0 / sqrt(ww);
            const R sc = (R)inv, arr = (R)(tot[nb + rr].x * inv), aii = (R)(tot[nb + rr].y * inv);
            const int ie = rr * N + e0 + eo;
            C<R> z = Zk[ie], w = Wk[ie], xx = a.x[ie], q = a.r[ie];
            z.x *= sc; z.y *= sc; w.x *= sc; w.y *= sc;
            xx.x += arr * z.x - aii * z.y;
            xx.y += arr * z.y + aii * z.x;
            q.x -= arr * w.x - aii * w.y;
            q.y -= arr * w.y + aii * w.x;
            Zk[ie] = z; Wk[ie] = w; a.x[ie] = xx; a.r[ie] = q;
        }
        __syncthreads();
        if (threadIdx.x < nb) {
            const int rr = threadIdx.x;
            if (act[rr]) {
                const double ww = tot[rr].x;
                if (!(ww > 0.0)) {
                    act[rr] = 0;
                } else {
                    const double ar = tot[nb + rr].x / sqrt(ww), ai = tot[nb + rr].y / sqrt(ww);
                    rn2[rr] -= ar * ar + ai * ai;
                    its[rr]++;
                    if (rn2[rr] <= stop[rr] || its[rr] >= a.maxiter) act[rr] = 0;
                }
            }
        }
        __syncthreads();
        ++k;
        if (k == a.restart) {
            // true residual r = b - A x for the right-hand sides still iterating
            bool any2 = false;
            for (int rr = 0; rr < nb; ++rr) any2 |= act[rr] != 0;
            if (any2) {
                __threadfence();
                grid.sync();
                apply_tasks<R, LT, NV>(a, a.r, a.x, N, s0, s1, act);
                zero_red(nb);
                for (int base = warp * 32; base < nitems; base += BCT) {
                    const int rr = (int)(base / Epad);
                    if (!act[rr]) continue;
                    const int eo = base - rr * Epad + lane;
                    double2 v = make_double2(0, 0);
                    if (eo < E) {
                        const int ie = rr * N + e0 + eo;
                        const C<R> bv = a.b[ie], ax = a.r[ie];
                        const C<R> q = mk<R>(bv.x - ax.x, bv.y - ax.y);
                        a.r[ie] = q;
                        v.x = (double)q.x * q.x + (double)q.y * q.y;
                    }
                    v = wsum(v);
                    if (lane == 0) red[warp][rr] = red[warp][rr] + v;
                }
                finish(nb);
                if (threadIdx.x < nb && act[threadIdx.x]) {
                    rn2[threadIdx.x] = tot[threadIdx.x].x;
                    if (rn2[threadIdx.x] <= stop[threadIdx.x]) act[threadIdx.x] = 0;
                }
                __syncthreads();
            }
            k = 0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int s = 0;
        for (int rr = 0; rr < nb; ++rr) s += its[rr];
        atomicAdd(a.iters, s);
    }
}

template <typename R, typename LT>
void launch_bt(dwf_ctx *c, const Level &L, const LT *Y, C<R> *x, const C<R> *b, int nb, C<R> *r, C<R> *Z, C<R> *W,
               double2 *part, int *iters, double tol, int maxiter, int restart) {
    BArgs<R, LT> a;
    a.Y = Y;
    a.nbr = L.nbr.as<int>();
    a.g = L.lg.g;
    a.b = b;
    a.x = x;
    a.r = r;
    a.Z = Z;
    a.W = W;
    a.part = part;
    a.tot = part + (size_t)MAXV * c->sm_count;
    a.tol = tol;
    a.maxiter = maxiter;
    a.restart = restart;
    a.nb = nb;
    a.iters = iters;
    void *kargs[] = {&a};
    const int n = L.lg.ncomp;
    DWF_REQUIRE(L.nbr.p, DWF_ESTATE, "coarse level without a neighbour table");
    DWF_REQUIRE((int64_t)L.lg.g.V * n * nb < ((int64_t)1 << 31), DWF_EINVAL,
                "batched coarse solve: nb coarse fields exceed 32-bit indexing");
    void *fn = nullptr;
    switch (n) {
        case 2: fn = (void *)coarse_gcr_batch_kernel<R, LT, 2>; break;
        case 4: fn = (void *)coarse_gcr_batch_kernel<R, LT, 4>; break;
        case 6: fn = (void *)coarse_gcr_batch_kernel<R, LT, 6>; break;
        case 8: fn = (void *)coarse_gcr_batch_kernel<R, LT, 8>; break;
        case 12: fn = (void *)coarse_gcr_batch_kernel<R, LT, 12>; break;
        case 16: fn = (void *)coarse_gcr_batch_kernel<R, LT, 16>; break;
        case 24: fn = (void *)coarse_gcr_batch_kernel<R, LT, 24>; break;
        case 32: fn = (void *)coarse_gcr_batch_kernel<R, LT, 32>; break;
        default: throw Error{DWF_EINVAL, "unsupported Nvec"};
    }
    int per_sm = 0;
    DWF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, BCT, 0));
    DWF_REQUIRE(per_sm >= 1, DWF_ECUDA, "batched coarse solver cannot be co-resident");
    // about four sites per CTA, at most one CTA per SM
    int64_t nblk = (L.lg.g.V + 3) / 4;
    nblk = std::max<int64_t>(1, std::min<int64_t>(nblk, c->sm_count));
    DWF_CUDA(coop_launch(c, fn, dim3((unsigned)nblk), dim3(BCT), kargs, 0));
    DWF_CHECK_LAUNCH();
}

}  // namespace

bool coarse_gcr_batch_ok(const Level &L, int restart, int nb) {
    return restart >= 1 && restart <= BMAXR && nb >= 1 && nb <= BMAXB;
}

// partial sums and totals; the tensor-core solver's two alternating buffers
// of FP32 partials (2 x (16 + 2) x 16 complex values per CTA, at most
// sm_count CTAs) take no more
size_t coarse_gcr_batch_part_bytes(dwf_ctx *c) { return sizeof(double2) * (size_t)MAXV * (c->sm_count + 1) + 256; }

template <typename R>
void coarse_gcr_fused_batch(dwf_ctx *c, const Level &L, C<R> *x, const C<R> *b, int nb, C<R> *r, C<R> *Z, C<R> *W,
                            double2 *part, int *iters, double tol, int maxiter, int restart) {
    DWF_REQUIRE(coarse_gcr_batch_ok(L, restart, nb), DWF_EINVAL, "batched coarse solve: restart <= 16, nb <= 16");
    if constexpr (std::is_same<R, float>::value) {
        if (coarse_gcr_tc_ok(c, L, restart, nb)) {
            coarse_gcr_tc(c, L, x, b, nb, r, Z, W, part, iters, tol, maxiter, restart);
            return;
        }
    }
    ProfScope ps(c, K_COARSE, nb);
    switch (L.yprec) {
        case DWF_F64: launch_bt<R, double2>(c, L, L.Y64.as<double2>(), x, b, nb, r, Z, W, part, iters, tol, maxiter, restart); break;
        case DWF_F32: launch_bt<R, float2>(c, L, L.Y32.as<float2>(), x, b, nb, r, Z, W, part, iters, tol, maxiter, restart); break;
        case DWF_BF16: launch_bt<R, __nv_bfloat162>(c, L, L.Y16.as<__nv_bfloat162>(), x, b, nb, r, Z, W, part, iters, tol, maxiter, restart); break;
        case DWF_F16: launch_bt<R, __half2>(c, L, L.Y16.as<__half2>(), x, b, nb, r, Z, W, part, iters, tol, maxiter, restart); break;
    }
}

template void coarse_gcr_fused_batch<float>(dwf_ctx *, const Level &, float2 *, const float2 *, int, float2 *, float2 *,
                                            float2 *, double2 *, int *, double, int, int);
template void coarse_gcr_fused_batch<double>(dwf_ctx *, const Level &, double2 *, const double2 *, int, double2 *,
                                             double2 *, double2 *, double2 *, int *, double, int, int);

}  // namespace dwf
