// Batched vector kernels: nrhs fields of n elements stored one after the
// other, blockIdx.y = right-hand side.  Every right-hand side has its own
// coefficients, read from device memory (scalar slots or coefficient
// arrays), and its own deterministic FP64-accumulated reductions.
#include "mg.cuh"

namespace dwf {

namespace {

constexpr int BT = 256;

template <typename T> struct RealB;
template <> struct RealB<float2> { using type = float; };
template <> struct RealB<double2> { using type = double; };

__device__ __forceinline__ double2 bsum(double2 v, double2 *sh) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x + 31) / 32) ? sh[threadIdx.x] : make_double2(0, 0);
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, o);
            v.y += __shfl_down_sync(0xffffffffu, v.y, o);
        }
    __syncthreads();
    return v;
}

// K complex reductions per right-hand side: out[base + r*stride + 2j (+1)];
// a real result (CPLX = false, K = 1) writes the single slot base + r*stride
template <int K, bool CPLX = true>
__device__ void finish_b(const double2 (&mine)[K], double2 *part, unsigned *count, double *s, int base, int stride) {
    __shared__ double2 sh[32];
    __shared__ bool last;
    const int r = blockIdx.y, nb = gridDim.x;
    double2 *pr = part + (size_t)r * K * nb;
    for (int j = 0; j < K; ++j) {
        double2 t = bsum(mine[j], sh);
        if (threadIdx.x == 0) pr[(size_t)j * nb + blockIdx.x] = t;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned ticket = atomicAdd(count + r, 1u);
        last = (ticket == nb - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int j = 0; j < K; ++j) {
        double2 v = make_double2(0, 0);
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            const volatile double *pp = reinterpret_cast<const volatile double *>(&pr[(size_t)j * nb + i]);
            v.x += pp[0];
            v.y += pp[1];
        }
        v = bsum(v, sh);
        if (threadIdx.x == 0) {
            s[base + r * stride + 2 * j] = v.x;
            if (CPLX) s[base + r * stride + 2 * j + 1] = v.y;
        }
    }
    if (threadIdx.x == 0) count[r] = 0u;
}

// s[base + r*stride] = |x_r|^2
template <typename T>
__global__ void __launch_bounds__(BT) norm2_b_kernel(const T *__restrict__ x, int64_t n, double2 *part, unsigned *count,
                                                     double *s, int base, int stride) {
    using A = typename RealB<T>::type;
    x += (size_t)blockIdx.y * n;
    A a = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T u = x[i];
        a += u.x * u.x + u.y * u.y;
    }
    double2 m[1] = {make_double2((double)a, 0.0)};
    finish_b<1, false>(m, part, count, s, base, stride);
}

// s[base + r*stride + 2j (+1)] = <V_j,r, w_r>, j < K (w read once)
template <typename T, int K> struct VArgs {
    const T *v[K];
};
template <typename T, int K>
__global__ void __launch_bounds__(BT) multidot_b_kernel(VArgs<T, K> va, const T *__restrict__ w, int64_t n,
                                                        double2 *part, unsigned *count, double *s, int base,
                                                        int stride) {
    using A = typename RealB<T>::type;
    const size_t off = (size_t)blockIdx.y * n;
    A ar[K], ai[K];
#pragma unroll
    for (int j = 0; j < K; ++j) ar[j] = ai[j] = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T y = w[off + i];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            T u = va.v[j][off + i];
            ar[j] += u.x * y.x + u.y * y.y;
            ai[j] += u.x * y.y - u.y * y.x;
        }
    }
    double2 m[K];
#pragma unroll
    for (int j = 0; j < K; ++j) m[j] = make_double2((double)ar[j], (double)ai[j]);
    finish_b<K>(m, part, count, s, base, stride);
}

// w_r += sgn * sum_j c_{r,j} V_j,r with c from slots s[base + r*stride + 2j]
template <typename T> struct MArgs {
    const T *v[32];
    int k;
};
template <typename T>
__global__ void multiaxpy_b_kernel(T *__restrict__ w, MArgs<T> a, const double *__restrict__ s, int base, int stride,
                                   double sgn, int64_t n) {
    using R = typename RealB<T>::type;
    const int r = blockIdx.y;
    const size_t off = (size_t)r * n;
    R cr[32], ci[32];
    for (int j = 0; j < a.k; ++j) {
        cr[j] = (R)(sgn * s[base + r * stride + 2 * j]);
        ci[j] = (R)(sgn * s[base + r * stride + 2 * j + 1]);
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v = w[off + i];
        for (int j = 0; j < a.k; ++j) {
            T u = a.v[j][off + i];
            v.x += cr[j] * u.x - ci[j] * u.y;
            v.y += cr[j] * u.y + ci[j] * u.x;
        }
        w[off + i] = v;
    }
}

// The CGNR step split so that every field is read once per iteration:
//   r:  a = s[izz] / s[iww]; r -= a w
//   px: a as above, b = s[inew] / s[izz]; x += a p; p = z + b p
//   x:  x += a p (the last iteration, whose residual is not needed)
template <typename T>
__global__ void cg_r_b_kernel(T *rout, const T *rin, const T *__restrict__ w, const double *__restrict__ s, int base,
                              int stride, int izz, int iww, int64_t n) {
    using R = typename RealB<T>::type;
    const int r = blockIdx.y;
    const size_t off = (size_t)r * n;
    const double ww = s[base + r * stride + iww];
    const R a = ww > 0.0 ? (R)(s[base + r * stride + izz] / ww) : R(0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T rv = rin[off + i];
        const T wv = w[off + i];
        rv.x -= a * wv.x;
        rv.y -= a * wv.y;
        rout[off + i] = rv;
    }
}
template <typename T>
__global__ void cg_px_b_kernel(T *__restrict__ x, T *pout, const T *pin, const T *__restrict__ z,
                               const double *__restrict__ s, int base, int stride, int izz, int iww, int inew,
                               int64_t n, int last, int xinit) {
    using R = typename RealB<T>::type;
    const int r = blockIdx.y;
    const size_t off = (size_t)r * n;
    const double ww = s[base + r * stride + iww], zz = s[base + r * stride + izz];
    const R a = ww > 0.0 ? (R)(zz / ww) : R(0);
    const R b = (!last && zz > 0.0) ? (R)(s[base + r * stride + inew] / zz) : R(0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T pv = pin[off + i];
        T xv;
        if (xinit) {
            xv.x = a * pv.x;
            xv.y = a * pv.y;
        } else {
            xv = x[off + i];
            xv.x += a * pv.x;
            xv.y += a * pv.y;
        }
        x[off + i] = xv;
        if (!last) {
            const T zv = z[off + i];
            pv.x = zv.x + b * pv.x;
            pv.y = zv.y + b * pv.y;
            pout[off + i] = pv;
        }
    }
}

// CGNR direction update with the solution update x += a p deferred: up to
// CG_MAXDEFER directions whose steps are not in x yet wait in buffers of
// their own, their steps in the scalar slots ia, ia+1, ...  a = zz/ww and
// b = z'z'/zz of the current iteration as in cg_px_b.
//   mode 0 (defer): pout = z + b pin; s[ia + NP] = a (pin joins the pending)
//   mode 1 (flush): x += sum_j s[ia + j] pend[j] + a pin; pout = z + b pin
//   mode 2 (flush, last iteration): x += sum_j s[ia + j] pend[j] + a pin
// pout may be one of the pending buffers (each element is read before it is written).
template <typename T> struct Pending {
    const T *p[CG_MAXDEFER];
};
template <typename T, int NP>
__global__ void cg_pxd_b_kernel(T *__restrict__ x, T *pout, const T *__restrict__ pin, Pending<T> pend,
                                const T *__restrict__ z, double *s, int base, int stride, int izz, int iww, int inew,
                                int ia, int64_t n, int mode) {
    using R = typename RealB<T>::type;
    const int r = blockIdx.y;
    const size_t off = (size_t)r * n;
    double *sr = s + base + (size_t)r * stride;
    const double ww = sr[iww], zz = sr[izz];
    const R a = ww > 0.0 ? (R)(zz / ww) : R(0);
    const R b = (mode != 2 && zz > 0.0) ? (R)(sr[inew] / zz) : R(0);
    R ap[NP > 0 ? NP : 1];
#pragma unroll
    for (int j = 0; j < NP; ++j) ap[j] = mode != 0 ? (R)sr[ia + j] : R(0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T pv = pin[off + i];
        if (mode != 0) {
            T xv = x[off + i];
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                const T qv = pend.p[j][off + i];
                xv.x += ap[j] * qv.x;
                xv.y += ap[j] * qv.y;
            }
            xv.x += a * pv.x;
            xv.y += a * pv.y;
            x[off + i] = xv;
        }
        if (mode != 2) {
            const T zv = z[off + i];
            pv.x = zv.x + b * pv.x;
            pv.y = zv.y + b * pv.y;
            pout[off + i] = pv;
        }
    }
    // a defer launch reads no pending step, so no CTA can see this slot change
    if (mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) sr[ia + NP] = (double)a;
}

// w_r *= sc[r];  res_r -= al[r] * w_r   (GCR direction normalisation and residual update)
template <typename T>
__global__ void gcr_wr_b_kernel(T *__restrict__ w, T *__restrict__ res, const double *__restrict__ sc,
                                const double2 *__restrict__ al, int64_t n) {
    using R = typename RealB<T>::type;
    const int r = blockIdx.y;
    const size_t off = (size_t)r * n;
    const R s = (R)sc[r], ar = (R)al[r].x, ai = (R)al[r].y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T wv = w[off + i], rv = res[off + i];
        wv.x *= s;
        wv.y *= s;
        rv.x -= ar * wv.x - ai * wv.y;
        rv.y -= ar * wv.y + ai * wv.x;
        w[off + i] = wv;
        res[off + i] = rv;
    }
}

// x_r += sum_j g[r*k + j] V_j,r (per-RHS coefficient arrays, k <= 32)
template <typename T>
__global__ void combo_b_kernel(T *__restrict__ x, MArgs<T> a, const double2 *__restrict__ g, int64_t n) {
    using R = typename RealB<T>::type;
    const int r = blockIdx.y;
    const size_t off = (size_t)r * n;
    R cr[32], ci[32];
    for (int j = 0; j < a.k; ++j) {
        cr[j] = (R)g[r * a.k + j].x;
        ci[j] = (R)g[r * a.k + j].y;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v = x[off + i];
        for (int j = 0; j < a.k; ++j) {
            T u = a.v[j][off + i];
            v.x += cr[j] * u.x - ci[j] * u.y;
            v.y += cr[j] * u.y + ci[j] * u.x;
        }
        x[off + i] = v;
    }
}

// x_r += sum_j g_j Z_j,r for the k (<= 32) stored normal-equations residuals
// z_0 .. z_{k-1} of k CGNR iterations, with g the solution's coefficients in
// that basis: x = sum_k a_k p_k and p_k = z_k + b_{k-1} p_{k-1} give
// g_{k-1} = a_{k-1}, g_j = a_j + b_j g_{j+1}, where a_j = |z_j|^2 / |w_j|^2
// and b_j = |z_{j+1}|^2 / |z_j|^2 come from the scalar slots zb + j and wb + j.
template <typename T>
__global__ void cg_combine_b_kernel(T *__restrict__ x, MArgs<T> a, const double *__restrict__ s, int base, int stride,
                                    int zb, int wb, int64_t n) {
    using R = typename RealB<T>::type;
    __shared__ R gam[32];
    const int r = blockIdx.y;
    const size_t off = (size_t)r * n;
    if (threadIdx.x == 0) {
        const double *sr = s + base + (size_t)r * stride;
        double g = 0.0;
        for (int j = a.k - 1; j >= 0; --j) {
            const double zz = sr[zb + j], ww = sr[wb + j];
            const double al = ww > 0.0 ? zz / ww : 0.0;
            const double be = (j + 1 < a.k && zz > 0.0) ? sr[zb + j + 1] / zz : 0.0;
            g = al + be * g;
            gam[j] = (R)g;
        }
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v = x[off + i];
#pragma unroll 8
        for (int j = 0; j < a.k; ++j) {
            const T u = a.v[j][off + i];
            v.x += gam[j] * u.x;
            v.y += gam[j] * u.y;
        }
        x[off + i] = v;
    }
}

// End of a chunk of m CGNR iterations k0 .. k0+m-1 that kept the residuals
// z_{k0+1} .. z_{k0+m-1} (and z_{k0+m} when the chunk is not the last) and
// carried w = D p by recursion.  With p_0 the chunk's first direction,
// p_t = z_t + b_{t-1} p_{t-1}:
//   x (+)= sum_t a_t p_t = G_0 p_0 + sum_{t=1}^{m-1} G_t z_t,
//          G_{m-1} = a_{m-1}, G_t = a_t + b_t G_{t+1};
//   p_0 <- p_m = P_0 p_0 + sum_{t=1}^{m} P_t z_t, P_m = 1, P_t = b_t P_{t+1}
// (the latter only with next).  a_t = |z_t|^2 / |w_t|^2 and
// b_t = |z_{t+1}|^2 / |z_t|^2 from the ring of scalar slots
// zb + (k0 + t) % rs and wb + (k0 + t) % rs.
template <typename T>
__global__ void cg_chunk_b_kernel(T *__restrict__ x, T *__restrict__ p, MArgs<T> z, const double *__restrict__ s,
                                  int base, int stride, int zb, int wb, int k0, int rs, int m, int next, int xinit,
                                  int64_t n) {
    using R = typename RealB<T>::type;
    __shared__ R G[33], P[33];
    const int r = blockIdx.y;
    const size_t off = (size_t)r * n;
    if (threadIdx.x == 0) {
        const double *sr = s + base + (size_t)r * stride;
        auto zz = [&](int t) { return sr[zb + (k0 + t) % rs]; };
        auto ww = [&](int t) { return sr[wb + (k0 + t) % rs]; };
        double g = 0.0, q = 1.0;
        if (next) P[m] = (R)1;
        for (int t = m - 1; t >= 0; --t) {
            const double zt = zz(t), wt = ww(t);
            const double al = wt > 0.0 ? zt / wt : 0.0;
            const bool have_b = t + 1 < m || next;
            const double be = (have_b && zt > 0.0) ? zz(t + 1) / zt : 0.0;
            g = al + (t + 1 < m ? be * g : 0.0);
            G[t] = (R)g;
            if (next) {
                q *= be;
                P[t] = (R)q;
            }
        }
    }
    __syncthreads();
    const int nz = next ? m : m - 1;  // z pointers: z_1 .. z_nz
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T pv = p[off + i];
        T xv = xinit ? T{0, 0} : x[off + i];
        T pn = next ? T{P[0] * pv.x, P[0] * pv.y} : T{0, 0};
        xv.x += G[0] * pv.x;
        xv.y += G[0] * pv.y;
#pragma unroll 8
        for (int t = 1; t <= nz; ++t) {
            const T u = z.v[t - 1][off + i];
            if (t < m) {
                xv.x += G[t] * u.x;
                xv.y += G[t] * u.y;
            }
            if (next) {
                pn.x += P[t] * u.x;
                pn.y += P[t] * u.y;
            }
        }
        x[off + i] = xv;
        if (next) p[off + i] = pn;
    }
}

dim3 grid_b(dwf_ctx *c, int64_t n, int nrhs, int cap_per_sm) {
    int64_t b = (n + BT - 1) / BT;
    int64_t cap = std::max<int64_t>(1, (int64_t)c->sm_count * cap_per_sm / std::max(1, nrhs));
    cap = std::min<int64_t>(cap, 1024);  // partial-sum buffers hold 1024 blocks per value
    return dim3((unsigned)std::max<int64_t>(1, std::min(b, cap)), (unsigned)nrhs);
}

}  // namespace

// Buffers of batched reductions: partial sums [nrhs][8][blocks] and counters.
void BatchScratch::ensure(int nrhs) {
    size_t need = sizeof(double2) * (size_t)nrhs * 8 * 1024;
    if (part.bytes < need) part.alloc(need);
    if (count.bytes < sizeof(unsigned) * (size_t)nrhs) {
        count.alloc(sizeof(unsigned) * (size_t)nrhs);
        DWF_CUDA(cudaMemset(count.p, 0, count.bytes));
    }
}

template <typename T> void norm2_b(dwf_ctx *c, BatchScratch &bs, int base, int stride, const T *x, int64_t n, int nrhs) {
    dim3 g = grid_b(c, n, nrhs, 8);
    norm2_b_kernel<T><<<g, BT, 0, c->stream>>>(x, n, bs.part.as<double2>(), bs.count.as<unsigned>(), c->scal.as<double>(),
                                               base, stride);
    DWF_CHECK_LAUNCH();
}

template <typename T>
void multidot_b(dwf_ctx *c, BatchScratch &bs, int base, int stride, T *const *V, int k, const T *w, int64_t n, int nrhs) {
    dim3 g = grid_b(c, n, nrhs, 8);
    for (int j0 = 0; j0 < k; j0 += 8) {
        int kk = std::min(8, k - j0);
#define MDB(K)                                                                                              \
    {                                                                                                       \
        VArgs<T, K> a;                                                                                      \
        for (int j = 0; j < K; ++j) a.v[j] = V[j0 + j];                                                     \
        multidot_b_kernel<T, K><<<g, BT, 0, c->stream>>>(a, w, n, bs.part.as<double2>(), bs.count.as<unsigned>(), \
                                                         c->scal.as<double>(), base + 2 * j0, stride);      \
    }
        switch (kk) {
            case 1: MDB(1) break;
            case 2: MDB(2) break;
            case 3: MDB(3) break;
            case 4: MDB(4) break;
            case 5: MDB(5) break;
            case 6: MDB(6) break;
            case 7: MDB(7) break;
            default: MDB(8) break;
        }
#undef MDB
        DWF_CHECK_LAUNCH();
    }
}

template <typename T>
void multiaxpy_b(dwf_ctx *c, T *w, T *const *V, int k, int base, int stride, double sgn, int64_t n, int nrhs) {
    dim3 g = grid_b(c, n, nrhs, 16);
    for (int j0 = 0; j0 < k; j0 += 32) {
        MArgs<T> a;
        a.k = std::min(32, k - j0);
        for (int j = 0; j < a.k; ++j) a.v[j] = V[j0 + j];
        multiaxpy_b_kernel<T><<<g, BT, 0, c->stream>>>(w, a, c->scal.as<double>(), base + 2 * j0, stride, sgn, n);
        DWF_CHECK_LAUNCH();
    }
}

template <typename T>
void cg_r_b(dwf_ctx *c, T *r, const T *rin, const T *w, int base, int stride, int izz, int iww, int64_t n, int nrhs) {
    dim3 g = grid_b(c, n, nrhs, 16);
    cg_r_b_kernel<T><<<g, BT, 0, c->stream>>>(r, rin, w, c->scal.as<double>(), base, stride, izz, iww, n);
    DWF_CHECK_LAUNCH();
}

template <typename T>
void cg_px_b(dwf_ctx *c, T *x, T *pout, const T *pin, const T *z, int base, int stride, int izz, int iww, int inew,
             int64_t n, int nrhs, bool last, bool xinit) {
    dim3 g = grid_b(c, n, nrhs, 16);
    cg_px_b_kernel<T><<<g, BT, 0, c->stream>>>(x, pout, pin, z, c->scal.as<double>(), base, stride, izz, iww, inew,
                                               n, last ? 1 : 0, xinit ? 1 : 0);
    DWF_CHECK_LAUNCH();
}

template <typename T>
void cg_pxd_b(dwf_ctx *c, T *x, T *pout, const T *pin, T *const *pend, int np, const T *z, int base, int stride,
              int izz, int iww, int inew, int ia, int64_t n, int nrhs, int mode) {
    DWF_REQUIRE(mode >= 0 && mode <= 2 && np >= 0 && np <= CG_MAXDEFER && !(mode == 0 && np == CG_MAXDEFER),
                DWF_EINVAL, "cg_pxd_b: mode or pending count");
    dim3 g = grid_b(c, n, nrhs, 16);
    Pending<T> pd{};
    for (int j = 0; j < np; ++j) pd.p[j] = pend[j];
    double *s = c->scal.as<double>();
#define PX(NP) cg_pxd_b_kernel<T, NP><<<g, BT, 0, c->stream>>>(x, pout, pin, pd, z, s, base, stride, izz, iww, inew, ia, \
                                                                n, mode)
    switch (np) {
        case 0: PX(0); break;
        case 1: PX(1); break;
        case 2: PX(2); break;
        default: PX(3); break;
    }
#undef PX
    DWF_CHECK_LAUNCH();
}

template <typename T>
void gcr_wr_b(dwf_ctx *c, T *w, T *res, const double *sc, const double2 *al, int64_t n, int nrhs) {
    dim3 g = grid_b(c, n, nrhs, 16);
    gcr_wr_b_kernel<T><<<g, BT, 0, c->stream>>>(w, res, sc, al, n);
    DWF_CHECK_LAUNCH();
}

template <typename T> void combo_b(dwf_ctx *c, T *x, T *const *V, int k, const double2 *g, int64_t n, int nrhs) {
    DWF_REQUIRE(k <= 32, DWF_EINVAL, "combo_b: at most 32 vectors");
    if (k == 0) return;
    dim3 gr = grid_b(c, n, nrhs, 16);
    MArgs<T> a;
    a.k = k;
    for (int j = 0; j < k; ++j) a.v[j] = V[j];
    combo_b_kernel<T><<<gr, BT, 0, c->stream>>>(x, a, g, n);
    DWF_CHECK_LAUNCH();
}

template <typename T>
void cg_combine_b(dwf_ctx *c, T *x, T *const *Z, int k, int base, int stride, int zb, int wb, int64_t n, int nrhs) {
    DWF_REQUIRE(k >= 1 && k <= 32, DWF_EINVAL, "cg_combine_b: 1 to 32 stored residuals");
    dim3 gr = grid_b(c, n, nrhs, 16);
    MArgs<T> a;
    a.k = k;
    for (int j = 0; j < k; ++j) a.v[j] = Z[j];
    cg_combine_b_kernel<T><<<gr, BT, 0, c->stream>>>(x, a, c->scal.as<double>(), base, stride, zb, wb, n);
    DWF_CHECK_LAUNCH();
}

template <typename T>
void cg_chunk_b(dwf_ctx *c, T *x, T *p, T *const *Z, int m, bool next, bool xinit, int base, int stride, int zb, int wb,
                int k0, int rs, int64_t n, int nrhs) {
    DWF_REQUIRE(m >= 1 && m <= 32 && rs > m, DWF_EINVAL, "cg_chunk_b: 1 to 32 iterations, slot ring longer than that");
    dim3 gr = grid_b(c, n, nrhs, 16);
    MArgs<T> a;
    a.k = next ? m : m - 1;
    for (int j = 0; j < a.k; ++j) a.v[j] = Z[j];
    cg_chunk_b_kernel<T><<<gr, BT, 0, c->stream>>>(x, p, a, c->scal.as<double>(), base, stride, zb, wb, k0, rs, m,
                                                   next ? 1 : 0, xinit ? 1 : 0, n);
    DWF_CHECK_LAUNCH();
}

#define INSTB(T)                                                                                            \
    template void norm2_b<T>(dwf_ctx *, BatchScratch &, int, int, const T *, int64_t, int);                  \
    template void multidot_b<T>(dwf_ctx *, BatchScratch &, int, int, T *const *, int, const T *, int64_t, int); \
    template void multiaxpy_b<T>(dwf_ctx *, T *, T *const *, int, int, int, double, int64_t, int);            \
    template void cg_r_b<T>(dwf_ctx *, T *, const T *, const T *, int, int, int, int, int64_t, int);          \
    template void cg_px_b<T>(dwf_ctx *, T *, T *, const T *, const T *, int, int, int, int, int, int64_t, int, bool, \
                             bool);                                                                            \
    template void cg_pxd_b<T>(dwf_ctx *, T *, T *, const T *, T *const *, int, const T *, int, int, int, int, int, \
                              int, int64_t, int, int);                                                         \
    template void cg_combine_b<T>(dwf_ctx *, T *, T *const *, int, int, int, int, int, int64_t, int);        \
    template void cg_chunk_b<T>(dwf_ctx *, T *, T *, T *const *, int, bool, bool, int, int, int, int, int, int,   \
                                int64_t, int);                                                                 \
    template void gcr_wr_b<T>(dwf_ctx *, T *, T *, const double *, const double2 *, int64_t, int);            \
    template void combo_b<T>(dwf_ctx *, T *, T *const *, int, const double2 *, int64_t, int);
INSTB(float2)
INSTB(double2)

}  // namespace dwf
