// Layout conversion between the canonical fermion layout (complex128,
// index ((s*V + site)*4 + spin)*3 + colour) and the internal s-fastest
// layout ((site*12 + spin*3 + colour)*Ls + s) in FP64 or FP32, plus the
// two-row FP32 link copy.
#include "dwf_internal.cuh"

namespace dwf {

namespace {

template <typename T>
__global__ void pack_kernel(T *__restrict__ out, const double2 *__restrict__ in, int64_t V, int Ls, int nrhs) {
    const int64_t field = V * 12 * Ls;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < field * nrhs;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i / field, e = i - r * field;
        int s = (int)(e % Ls);
        int64_t sc = e / Ls;               // site*12 + comp
        int64_t site = sc / 12;
        int comp = (int)(sc - site * 12);
        out[i] = cvt<T, double2>(in[r * field + ((int64_t)s * V + site) * 12 + comp]);
    }
}

template <typename T>
__global__ void unpack_kernel(double2 *__restrict__ out, const T *__restrict__ in, int64_t V, int Ls, int nrhs) {
    const int64_t field = V * 12 * Ls;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < field * nrhs;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i / field, e = i - r * field;
        int s = (int)(e % Ls);
        int64_t sc = e / Ls;
        int64_t site = sc / 12;
        int comp = (int)(sc - site * 12);
        out[r * field + ((int64_t)s * V + site) * 12 + comp] = cvt<double2, T>(in[i]);
    }
}

__global__ void links32_kernel(float2 *__restrict__ out, const double2 *__restrict__ U, int64_t nlinks) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlinks * 6;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = i / 6;
        int e = (int)(i - l * 6);
        out[i] = cvt<float2, double2>(U[l * 9 + e]);
    }
}

unsigned grid_for(dwf_ctx *c, int64_t n) {
    int64_t b = (n + 255) / 256;
    int64_t cap = (int64_t)c->sm_count * 32;
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

void pack(dwf_ctx *c, void *internal, const double2 *canonical, dwf_prec prec, int nrhs) {
    int64_t n = c->g.V * 12 * c->g.Ls * nrhs;
    if (prec == DWF_F64)
        pack_kernel<double2><<<grid_for(c, n), 256, 0, c->stream>>>((double2 *)internal, canonical, c->g.V, c->g.Ls, nrhs);
    else
        pack_kernel<float2><<<grid_for(c, n), 256, 0, c->stream>>>((float2 *)internal, canonical, c->g.V, c->g.Ls, nrhs);
    DWF_CHECK_LAUNCH();
}

void unpack(dwf_ctx *c, double2 *canonical, const void *internal, dwf_prec prec, int nrhs) {
    int64_t n = c->g.V * 12 * c->g.Ls * nrhs;
    if (prec == DWF_F64)
        unpack_kernel<double2><<<grid_for(c, n), 256, 0, c->stream>>>(canonical, (const double2 *)internal, c->g.V, c->g.Ls, nrhs);
    else
        unpack_kernel<float2><<<grid_for(c, n), 256, 0, c->stream>>>(canonical, (const float2 *)internal, c->g.V, c->g.Ls, nrhs);
    DWF_CHECK_LAUNCH();
}

void pack_links(dwf_ctx *c, const double2 *U) {
    int64_t nl = c->g.V * 4;
    links32_kernel<<<grid_for(c, nl * 6), 256, 0, c->stream>>>(c->U32.as<float2>(), U, nl);
    DWF_CHECK_LAUNCH();
}

}  // namespace dwf
