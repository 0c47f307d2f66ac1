// The fused coarsest-level GCR on the squared operator's 33-point coarse
// stencil P^+ D^+ D P (Sec. 4), in a translation unit of its own so that the
// two stencil sizes compile in parallel.
#include "coarse_gcr_kernel.cuh"

namespace dwf {

template <typename R>
void coarse_gcr_launch_squared(dwf_ctx *c, const Level &L, C<R> *x, const C<R> *b, C<R> *r, C<R> *Z, C<R> *W,
                               double2 *part, int *iters, double tol, int maxiter, int restart) {
    switch (L.yprec) {
        case DWF_F64: launch_t<R, double2, 33>(c, L, L.Y64.as<double2>(), x, b, r, Z, W, part, iters, tol, maxiter, restart); break;
        case DWF_F32: launch_t<R, float2, 33>(c, L, L.Y32.as<float2>(), x, b, r, Z, W, part, iters, tol, maxiter, restart); break;
        case DWF_BF16: launch_t<R, __nv_bfloat162, 33>(c, L, L.Y16.as<__nv_bfloat162>(), x, b, r, Z, W, part, iters, tol, maxiter, restart); break;
        case DWF_F16: launch_t<R, __half2, 33>(c, L, L.Y16.as<__half2>(), x, b, r, Z, W, part, iters, tol, maxiter, restart); break;
    }
}

template void coarse_gcr_launch_squared<double>(dwf_ctx *, const Level &, double2 *, const double2 *, double2 *,
                                                double2 *, double2 *, double2 *, int *, double, int, int);
template void coarse_gcr_launch_squared<float>(dwf_ctx *, const Level &, float2 *, const float2 *, float2 *, float2 *,
                                               float2 *, double2 *, int *, double, int, int);

}  // namespace dwf
