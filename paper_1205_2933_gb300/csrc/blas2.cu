// Vector updates with host-side coefficients, and the device Philox
// generator of random start vectors.
#include "mg.cuh"

namespace dwf {

namespace {

// Arithmetic in the storage precision: FP32 fields are updated with FP32
// FMAs (GB300's FP64 rate is a small fraction of its FP32 rate).
template <typename T> struct Real;
template <> struct Real<double2> { using type = double; };
template <> struct Real<float2> { using type = float; };

template <typename T>
__global__ void caxpy_kernel(T *__restrict__ y, double2 ad, const T *__restrict__ x, int64_t n) {
    using R = typename Real<T>::type;
    const R ar = (R)ad.x, ai = (R)ad.y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T xv = x[i], yv = y[i];
        yv.x += ar * xv.x - ai * xv.y;
        yv.y += ar * xv.y + ai * xv.x;
        y[i] = yv;
    }
}

template <typename T>
__global__ void cxpay_kernel(T *__restrict__ y, double2 ad, const T *__restrict__ x, int64_t n) {
    using R = typename Real<T>::type;
    const R ar = (R)ad.x, ai = (R)ad.y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T xv = x[i], yv = y[i];
        T o;
        o.x = xv.x + ar * yv.x - ai * yv.y;
        o.y = xv.y + ar * yv.y + ai * yv.x;
        y[i] = o;
    }
}

template <typename T>
__global__ void rscale_kernel(T *__restrict__ x, double ad, int64_t n) {
    using R = typename Real<T>::type;
    const R a = (R)ad;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v = x[i];
        v.x *= a;
        v.y *= a;
        x[i] = v;
    }
}

template <typename T, typename U>
__global__ void caxpy_mixed_kernel(T *__restrict__ y, double2 a, const U *__restrict__ x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 xv = cvt<double2, U>(x[i]), yv = cvt<double2, T>(y[i]);
        yv.x += a.x * xv.x - a.y * xv.y;
        yv.y += a.x * xv.y + a.y * xv.x;
        y[i] = cvt<T, double2>(yv);
    }
}

template <typename T> struct MultiArgs {
    const T *p[32];
    double2 b[32];
    int k;
};

template <typename T>
__global__ void multiaxpy_kernel(T *__restrict__ w, MultiArgs<T> a, int64_t n) {
    using R = typename Real<T>::type;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v = w[i];
        for (int j = 0; j < a.k; ++j) {
            T u = a.p[j][i];
            const R br = (R)a.b[j].x, bi = (R)a.b[j].y;
            v.x += br * u.x - bi * u.y;
            v.y += br * u.y + bi * u.x;
        }
        w[i] = v;
    }
}

// Solver updates whose coefficients stay in device scalar slots (no host
// round trip).  s[] is the context's scalar array.
//   cg_xr:  a = s[izz] / s[iww] (0 if s[iww] <= 0); x += a p; r -= a w
//   cg_p:   b = s[inew] / s[iold] (0 if s[iold] <= 0); p = z + b p
template <typename T>
__global__ void cg_xr_kernel(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p, const T *__restrict__ w,
                             const double *__restrict__ s, int izz, int iww, int64_t n) {
    using R = typename Real<T>::type;
    const double ww = s[iww];
    const R a = ww > 0.0 ? (R)(s[izz] / ww) : R(0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T pv = p[i], wv = w[i], xv = x[i], rv = r[i];
        xv.x += a * pv.x;
        xv.y += a * pv.y;
        rv.x -= a * wv.x;
        rv.y -= a * wv.y;
        x[i] = xv;
        r[i] = rv;
    }
}

template <typename T>
__global__ void cg_p_kernel(T *__restrict__ p, const T *__restrict__ z, const double *__restrict__ s, int inew,
                            int iold, int64_t n) {
    using R = typename Real<T>::type;
    const double old = s[iold];
    const R bta = old > 0.0 ? (R)(s[inew] / old) : R(0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T pv = p[i], zv = z[i];
        pv.x = zv.x + bta * pv.x;
        pv.y = zv.y + bta * pv.y;
        p[i] = pv;
    }
}

// w += sum_j c_j V_j with c_j = sgn * (s[ibase + 2j], s[ibase + 2j + 1])
template <typename T>
__global__ void multiaxpy_dev_kernel(T *__restrict__ w, MultiArgs<T> a, const double *__restrict__ s, int ibase,
                                     double sgn, int64_t n) {
    using R = typename Real<T>::type;
    R cr[32], ci[32];
    for (int j = 0; j < a.k; ++j) {
        cr[j] = (R)(sgn * s[ibase + 2 * j]);
        ci[j] = (R)(sgn * s[ibase + 2 * j + 1]);
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v = w[i];
        for (int j = 0; j < a.k; ++j) {
            T u = a.p[j][i];
            v.x += cr[j] * u.x - ci[j] * u.y;
            v.y += cr[j] * u.y + ci[j] * u.x;
        }
        w[i] = v;
    }
}

// GCR step with device coefficients: ww = s[iww] = |w|^2, (s[ia], s[ia+1]) =
// <w, r>.  w, z are normalised by 1/|w|; x += al z; r -= al w with
// al = <w, r> / |w| (the coefficient of the normalised direction).
template <typename T>
__global__ void gcr_step_kernel(T *__restrict__ x, T *__restrict__ r, T *__restrict__ z, T *__restrict__ w,
                                const double *__restrict__ s, int iww, int ia, int64_t n) {
    using R = typename Real<T>::type;
    const double ww = s[iww];
    const double inv = ww > 0.0 ? 1.0 / sqrt(ww) : 0.0;
    const R sc = (R)inv;
    const R ar = (R)(s[ia] * inv), ai = (R)(s[ia + 1] * inv);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T zv = z[i], wv = w[i], xv = x[i], rv = r[i];
        zv.x *= sc; zv.y *= sc;
        wv.x *= sc; wv.y *= sc;
        xv.x += ar * zv.x - ai * zv.y;
        xv.y += ar * zv.y + ai * zv.x;
        rv.x -= ar * wv.x - ai * wv.y;
        rv.y -= ar * wv.y + ai * wv.x;
        z[i] = zv;
        w[i] = wv;
        x[i] = xv;
        r[i] = rv;
    }
}

// Philox-4x32-10 (Salmon et al., SC'11) and Box-Muller, matching the host
// input generator's addressing: key (seed, stream), counter (i, 0, 0, i>>32).
__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__global__ void gauss_kernel(double2 *__restrict__ out, int nfields, int64_t nelem, int Ls, int64_t V, int canon,
                             uint32_t seed, uint32_t stream) {
    const int64_t total = nelem * nfields;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = i / nelem, e = i - j * nelem;
        int64_t idx = i;
        if (canon) {  // internal (site*12 + comp)*Ls + s  ->  canonical (s*V + site)*12 + comp
            int s = (int)(e % Ls);
            int64_t sc = e / Ls;
            int64_t site = sc / 12;
            int comp = (int)(sc - site * 12);
            idx = j * nelem + ((int64_t)s * V + site) * 12 + comp;
        }
        uint32_t c[4] = {(uint32_t)idx, 0u, 0u, (uint32_t)(idx >> 32)};
        philox(c, seed, stream);
        const double inv53 = 1.0 / 9007199254740992.0;
        double u0 = ((double)(c[0] >> 5) * 67108864.0 + (double)(c[1] >> 6) + 0.5) * inv53;
        double u1 = ((double)(c[2] >> 5) * 67108864.0 + (double)(c[3] >> 6) + 0.5) * inv53;
        double r = sqrt(-2.0 * log(u0));
        double th = 6.283185307179586476925286766559 * u1;
        out[i] = make_double2(r * cos(th), r * sin(th));
    }
}

unsigned blocks_for(dwf_ctx *c, int64_t n) {
    int64_t b = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)c->sm_count * 16));
}

}  // namespace

template <typename T> void caxpy(dwf_ctx *c, T *y, double2 a, const T *x, int64_t n) {
    caxpy_kernel<T><<<blocks_for(c, n), 256, 0, c->stream>>>(y, a, x, n);
    DWF_CHECK_LAUNCH();
}
template <typename T> void cxpay(dwf_ctx *c, T *y, double2 a, const T *x, int64_t n) {
    cxpay_kernel<T><<<blocks_for(c, n), 256, 0, c->stream>>>(y, a, x, n);
    DWF_CHECK_LAUNCH();
}
template <typename T> void rscale(dwf_ctx *c, T *x, double a, int64_t n) {
    rscale_kernel<T><<<blocks_for(c, n), 256, 0, c->stream>>>(x, a, n);
    DWF_CHECK_LAUNCH();
}
template <typename T, typename U> void caxpy_mixed(dwf_ctx *c, T *y, double2 a, const U *x, int64_t n) {
    caxpy_mixed_kernel<T, U><<<blocks_for(c, n), 256, 0, c->stream>>>(y, a, x, n);
    DWF_CHECK_LAUNCH();
}
template <typename T> void multiaxpy(dwf_ctx *c, T *w, const double2 *beta, T *const *V, int k, int64_t n) {
    DWF_REQUIRE(k <= 32, DWF_EINVAL, "multiaxpy: at most 32 vectors");
    if (k == 0) return;
    MultiArgs<T> a;
    for (int j = 0; j < k; ++j) {
        a.p[j] = V[j];
        a.b[j] = beta[j];
    }
    a.k = k;
    multiaxpy_kernel<T><<<blocks_for(c, n), 256, 0, c->stream>>>(w, a, n);
    DWF_CHECK_LAUNCH();
}
template <typename T> void cg_xr(dwf_ctx *c, T *x, T *r, const T *p, const T *w, int izz, int iww, int64_t n) {
    cg_xr_kernel<T><<<blocks_for(c, n), 256, 0, c->stream>>>(x, r, p, w, c->scal.as<double>(), izz, iww, n);
    DWF_CHECK_LAUNCH();
}
template <typename T> void cg_p(dwf_ctx *c, T *p, const T *z, int inew, int iold, int64_t n) {
    cg_p_kernel<T><<<blocks_for(c, n), 256, 0, c->stream>>>(p, z, c->scal.as<double>(), inew, iold, n);
    DWF_CHECK_LAUNCH();
}
template <typename T> void multiaxpy_dev(dwf_ctx *c, T *w, T *const *V, int k, int ibase, double sgn, int64_t n) {
    for (int j0 = 0; j0 < k; j0 += 32) {
        MultiArgs<T> a;
        a.k = std::min(32, k - j0);
        for (int j = 0; j < a.k; ++j) {
            a.p[j] = V[j0 + j];
            a.b[j] = make_double2(0, 0);
        }
        multiaxpy_dev_kernel<T><<<blocks_for(c, n), 256, 0, c->stream>>>(w, a, c->scal.as<double>(), ibase + 2 * j0,
                                                                          sgn, n);
        DWF_CHECK_LAUNCH();
    }
}
template <typename T> void gcr_step(dwf_ctx *c, T *x, T *r, T *z, T *w, int iww, int ia, int64_t n) {
    gcr_step_kernel<T><<<blocks_for(c, n), 256, 0, c->stream>>>(x, r, z, w, c->scal.as<double>(), iww, ia, n);
    DWF_CHECK_LAUNCH();
}

template <typename T> void gauss_fill(dwf_ctx *c, double2 *out, int nfields, int64_t nelem, int Ls, int64_t V,
                                      bool canonical_fine, uint32_t seed, uint32_t stream) {
    gauss_kernel<<<blocks_for(c, nelem * nfields), 256, 0, c->stream>>>(out, nfields, nelem, Ls, V,
                                                                        canonical_fine ? 1 : 0, seed, stream);
    DWF_CHECK_LAUNCH();
}

template void caxpy<double2>(dwf_ctx *, double2 *, double2, const double2 *, int64_t);
template void caxpy<float2>(dwf_ctx *, float2 *, double2, const float2 *, int64_t);
template void cxpay<double2>(dwf_ctx *, double2 *, double2, const double2 *, int64_t);
template void cxpay<float2>(dwf_ctx *, float2 *, double2, const float2 *, int64_t);
template void rscale<double2>(dwf_ctx *, double2 *, double, int64_t);
template void rscale<float2>(dwf_ctx *, float2 *, double, int64_t);
template void caxpy_mixed<double2, float2>(dwf_ctx *, double2 *, double2, const float2 *, int64_t);
template void caxpy_mixed<double2, double2>(dwf_ctx *, double2 *, double2, const double2 *, int64_t);
template void multiaxpy<double2>(dwf_ctx *, double2 *, const double2 *, double2 *const *, int, int64_t);
template void multiaxpy<float2>(dwf_ctx *, float2 *, const double2 *, float2 *const *, int, int64_t);
template void cg_xr<double2>(dwf_ctx *, double2 *, double2 *, const double2 *, const double2 *, int, int, int64_t);
template void cg_xr<float2>(dwf_ctx *, float2 *, float2 *, const float2 *, const float2 *, int, int, int64_t);
template void cg_p<double2>(dwf_ctx *, double2 *, const double2 *, int, int, int64_t);
template void cg_p<float2>(dwf_ctx *, float2 *, const float2 *, int, int, int64_t);
template void multiaxpy_dev<double2>(dwf_ctx *, double2 *, double2 *const *, int, int, double, int64_t);
template void multiaxpy_dev<float2>(dwf_ctx *, float2 *, float2 *const *, int, int, double, int64_t);
template void gcr_step<double2>(dwf_ctx *, double2 *, double2 *, double2 *, double2 *, int, int, int64_t);
template void gcr_step<float2>(dwf_ctx *, float2 *, float2 *, float2 *, float2 *, int, int, int64_t);
template void gauss_fill<double2>(dwf_ctx *, double2 *, int, int64_t, int, int64_t, bool, uint32_t, uint32_t);

}  // namespace dwf
