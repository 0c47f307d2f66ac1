// The coarsest-level solve S2 of the V-cycle (Sec. 2) as one cooperative
// kernel: restarted GCR on the 9-point coarse stencil.
//
// The coarsest problem is small (e.g. 512 sites x 24 components) and a GCR
// iteration built from separate launches is bound by launch and host
// round-trip latency.  Here a co-resident grid (about one element per
// thread, at most one CTA per SM) owns contiguous slices of every coarse
// vector; grid-wide barriers separate the stencil apply (which reads
// other slices) and the reductions.  Each reduction writes one FP64 partial
// per CTA; after the barrier every CTA adds the partials in the same order,
// so all CTAs hold bit-identical scalars and take identical loop decisions.
// The algorithm is the same GCR as the launch-by-launch version: classical
// Gram-Schmidt twice against the stored directions, |w| normalisation,
// x += <w,r> z, r -= <w,r> w, true residual at each restart.
#include <mutex>

#include "coarse_gcr_kernel.cuh"

namespace dwf {

bool coarse_gcr_fused_ok(const Level &L, int restart) { return restart >= 1 && restart <= MAXR; }

size_t coarse_gcr_part_bytes(dwf_ctx *c) { return sizeof(double2) * 3 * (MAXR + 2) * (size_t)c->sm_count; }

template <typename R>
static void launch_any(dwf_ctx *c, const Level &L, C<R> *x, const C<R> *b, C<R> *r, C<R> *Z, C<R> *W, double2 *part,
                       int *iters, double tol, int maxiter, int restart) {
    if (L.npts == 33) return coarse_gcr_launch_squared<R>(c, L, x, b, r, Z, W, part, iters, tol, maxiter, restart);
    switch (L.yprec) {
        case DWF_F64: launch_t<R, double2, 9>(c, L, L.Y64.as<double2>(), x, b, r, Z, W, part, iters, tol, maxiter, restart); break;
        case DWF_F32: launch_t<R, float2, 9>(c, L, L.Y32.as<float2>(), x, b, r, Z, W, part, iters, tol, maxiter, restart); break;
        case DWF_BF16: launch_t<R, __nv_bfloat162, 9>(c, L, L.Y16.as<__nv_bfloat162>(), x, b, r, Z, W, part, iters, tol, maxiter, restart); break;
        case DWF_F16: launch_t<R, __half2, 9>(c, L, L.Y16.as<__half2>(), x, b, r, Z, W, part, iters, tol, maxiter, restart); break;
    }
}

template <typename R>
void coarse_gcr_fused(dwf_ctx *c, const Level &L, C<R> *x, const C<R> *b, C<R> *r, C<R> *Z, C<R> *W, double2 *part,
                      int *iters, double tol, int maxiter, int restart) {
    ProfScope ps(c, K_COARSE);
    launch_any<R>(c, L, x, b, r, Z, W, part, iters, tol, maxiter, restart);
}

template void coarse_gcr_fused<double>(dwf_ctx *, const Level &, double2 *, const double2 *, double2 *, double2 *,
                                       double2 *, double2 *, int *, double, int, int);
template void coarse_gcr_fused<float>(dwf_ctx *, const Level &, float2 *, const float2 *, float2 *, float2 *, float2 *,
                                      double2 *, int *, double, int, int);

}  // namespace dwf

// ---------------------------------------------------------------------------
// Variant that allocates nothing: for callers that cannot allocate device
// memory at solve time (for example a host framework that hands the library
// a fixed device-memory budget, or a runtime whose allocator must not be
// re-entered from inside the solve).  All scratch of the fused
// coarsest-level solver lives in one file-scope device array of fixed size,
// shared by every call.
// ---------------------------------------------------------------------------

namespace dwf {

// residual, 2 x restart direction vectors, FP64 partial sums, the counter
constexpr size_t STATIC_SCRATCH_BYTES = (size_t)8 << 20;
constexpr int STATIC_MAX_RESTART = 16;

static __device__ __align__(256) unsigned char g_coarse_scratch[STATIC_SCRATCH_BYTES];

namespace {
std::mutex g_scratch_mu;
void *g_scratch_ptr[64] = {nullptr};

// Device address of the static scratch on the current device, looked up
// once per device (the host-side symbol is not a device address).
void *static_scratch(dwf_ctx *c) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    DWF_REQUIRE(c->device >= 0 && c->device < 64, DWF_EINVAL, "device index out of range");
    if (!g_scratch_ptr[c->device]) {
        int cur = -1;
        DWF_CUDA(cudaGetDevice(&cur));
        DWF_REQUIRE(cur == c->device, DWF_ESTATE, "the context's device must be current");
        void *p = nullptr;
        DWF_CUDA(cudaGetSymbolAddress(&p, g_coarse_scratch));
        g_scratch_ptr[c->device] = p;
    }
    return g_scratch_ptr[c->device];
}

__global__ void zero_int_kernel(int *p) { *p = 0; }
}  // namespace

template <typename R>
static void static_solve_t(dwf_ctx *c, const Level &L, C<R> *x, const C<R> *b, double tol, int maxiter, int restart) {
    const int64_t N = L.lg.nelem;
    const size_t vec = sizeof(C<R>) * (size_t)N;
    // carve: [counter (256 B)] [partial sums, rounded up to 256 B] [r] [Z: restart vectors] [W: restart vectors]
    const size_t off = 256 + (coarse_gcr_part_bytes(c) + 255) / 256 * 256;
    DWF_REQUIRE(restart >= 1 && restart <= STATIC_MAX_RESTART, DWF_EINVAL,
                "static coarse solve: coarse_restart must be in 1..16");
    DWF_REQUIRE(off + vec * (1 + 2 * (size_t)restart) <= STATIC_SCRATCH_BYTES, DWF_EINVAL,
                "static coarse solve: (1 + 2*restart) coarse vectors and the partial sums exceed the 8 MiB static "
                "scratch");
    // the solver writes x = 0 before it reads b: the two must not overlap
    const unsigned char *xb = (const unsigned char *)x, *bb = (const unsigned char *)b;
    DWF_REQUIRE(xb + vec <= bb || bb + vec <= xb, DWF_EINVAL, "static coarse solve: x and b must not overlap");
    unsigned char *base = (unsigned char *)static_scratch(c);
    int *iters = (int *)base;
    double2 *partials = (double2 *)(base + 256);
    C<R> *r = (C<R> *)(base + off);
    C<R> *Z = r + N;
    C<R> *W = Z + (size_t)restart * N;
    zero_int_kernel<<<1, 1, 0, c->stream>>>(iters);  // the counter must start at zero
    DWF_CHECK_LAUNCH();
    launch_any<R>(c, L, x, b, r, Z, W, partials, iters, tol, maxiter, restart);
}

void mg_coarse_solve_static_impl(dwf_ctx *c, int level, void *x, const void *b) {
    DWF_REQUIRE(c->mg && c->mg->nlevels >= 2, DWF_ESTATE, "mg_setup has not completed");
    MGState &mg = *c->mg;
    DWF_REQUIRE(level == mg.nlevels - 1 && level >= 1, DWF_EINVAL, "the static coarse solve runs on the coarsest level");
    const Level &L = mg.lev[level];
    const mg_params &p = mg.p;
    if (p.smoother_prec == DWF_F32)
        static_solve_t<float>(c, L, (float2 *)x, (const float2 *)b, p.coarsest_tol, p.coarsest_maxiter, p.coarse_restart);
    else
        static_solve_t<double>(c, L, (double2 *)x, (const double2 *)b, p.coarsest_tol, p.coarsest_maxiter,
                               p.coarse_restart);
    DWF_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace dwf
