// Internal declarations of the dwfmg library (GB300, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <array>
#include <string>
#include <vector>

#include "dwfmg.h"

namespace dwf {

// ---------------------------------------------------------------------------
// Complex arithmetic on CUDA vector types
// ---------------------------------------------------------------------------
template <typename R> struct cplx_t;
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<float> { using type = float2; };
template <typename R> using C = typename cplx_t<R>::type;

template <typename R> __host__ __device__ __forceinline__ C<R> mk(R re, R im) { C<R> z; z.x = re; z.y = im; return z; }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__host__ __device__ __forceinline__ double2 conj2(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }
// i * a
template <typename T> __host__ __device__ __forceinline__ T mul_i(T a) { T r; r.x = -a.y; r.y = a.x; return r; }
// acc += a * b
template <typename T> __host__ __device__ __forceinline__ void cfma(T &acc, T a, T b) {
    acc.x += a.x * b.x - a.y * b.y;
    acc.y += a.x * b.y + a.y * b.x;
}
// acc += conj(a) * b
template <typename T> __host__ __device__ __forceinline__ void cfmac(T &acc, T a, T b) {
    acc.x += a.x * b.x + a.y * b.y;
    acc.y += a.x * b.y - a.y * b.x;
}

template <typename TO, typename TI> __host__ __device__ __forceinline__ TO cvt(TI a);
template <> __host__ __device__ __forceinline__ double2 cvt<double2, double2>(double2 a) { return a; }
template <> __host__ __device__ __forceinline__ float2 cvt<float2, float2>(float2 a) { return a; }
template <> __host__ __device__ __forceinline__ double2 cvt<double2, float2>(float2 a) { return make_double2(a.x, a.y); }
template <> __host__ __device__ __forceinline__ float2 cvt<float2, double2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
struct Error {
    dwf_status st;
    std::string msg;
};

#define DWF_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            throw ::dwf::Error{e_ == cudaErrorMemoryAllocation ? DWF_ENOMEM : DWF_ECUDA,       \
                               std::string(#call) + ": " + cudaGetErrorString(e_)};           \
    } while (0)

void note_launch();
void note_launches(unsigned long long n);  // kernels launched by a replayed graph
#define DWF_CHECK_LAUNCH()               \
    do {                                 \
        DWF_CUDA(cudaGetLastError());    \
        ::dwf::note_launch();            \
    } while (0)

#define DWF_REQUIRE(cond, code, text)                                                         \
    do {                                                                                      \
        if (!(cond)) throw ::dwf::Error{code, text};                                          \
    } while (0)

// Owned device buffer.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    explicit DevBuf(size_t n) { alloc(n); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t n) {
        release();
        if (n) DWF_CUDA(cudaMalloc(&p, n));
        bytes = n;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

// ---------------------------------------------------------------------------
// Lattice geometry shared by kernels
// ---------------------------------------------------------------------------
struct Geom {
    int L[4];      // X, Y, Z, T
    int Ls;        // fifth extent (1 on coarse levels)
    int64_t V;     // 4D volume
    int ap;        // antiperiodic in t
};

__host__ __device__ __forceinline__ void site_coords(const Geom &g, int64_t site, int c[4]) {
    c[0] = (int)(site % g.L[0]);
    site /= g.L[0];
    c[1] = (int)(site % g.L[1]);
    site /= g.L[1];
    c[2] = (int)(site % g.L[2]);
    c[3] = (int)(site / g.L[2]);
}
__host__ __device__ __forceinline__ int64_t site_index(const Geom &g, const int c[4]) {
    return (((int64_t)c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.L[0] + c[0];
}

// Device scalar slots used by solver kernels (coefficients stay on the GPU).
constexpr int NSCALAR = 8192;

struct MGState;

// Serialises the cooperative launches of the member contexts of a batch
// (each waits for the previous one to finish on the GPU).
struct CoopGate;
// cudaLaunchCooperativeKernel on c->stream, through c->gate when c belongs to a batch
cudaError_t coop_launch(dwf_ctx *c, const void *fn, dim3 grid, dim3 block, void **args, size_t smem);

// Kernel classes timed by the optional event profiler (see dwf_profile).
enum KernelClass {
    K_DSLASH_F64 = 0,
    K_DSLASH_F32 = 1,
    K_RESTRICT = 2,
    K_PROLONG = 3,
    K_COARSE = 4,
    K_DSLASH_F32_Z = 5,  // FP32 D or D^+ that reads a second field in its epilogue: b - D x, z - a D^+ w
    K_NCLASS = 6
};

struct ProfRecord {
    int cls;
    cudaEvent_t a, b;  // null for a launch inside a replayed graph: ms holds its time
    int units;         // fields (right-hand sides) the bracketed launch processed
    float ms;
};

}  // namespace dwf

// The opaque context of the C ABI.
struct dwf_ctx {
    dwf::Geom g;
    double M5, mf;
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 0;
    dwf_status sticky = DWF_OK;
    // links: FP64 full 3x3 [V][4][3][3]; FP32 two rows [V][4][2][3]
    dwf::DevBuf U64, U32;
    // device scalars (double), pinned host mirror
    dwf::DevBuf scal;
    double *hscal = nullptr;
    // reduction partial sums + completion counter
    dwf::DevBuf red_part, red_count;
    // per-CTA partial sums of the Dslash's fused output norms
    dwf::DevBuf dn_part;
    dwf::MGState *mg = nullptr;
    // error word of the tensor-core coarse solves (device int, owned by the
    // context: the solves' scratch is freed before the word is read back)
    dwf::DevBuf tc_err;
    bool tc_used = false;
    dwf::DevBuf tc_trial;  // iteration counter of the tensor-core solver's tuning trials
    // grid the tensor-core solver picked by timing, per (coarse sites, Nvec, batch width)
    std::vector<std::array<int64_t, 4>> tc_grid;
    // A batch of independent lattices (dwf_create with nlat > 1): one member
    // context per lattice, each on a stream of its own; the batch context
    // itself holds no lattice.  Cooperative launches of all members pass
    // through one gate so that two grids that each fill the GPU never wait
    // on one another.
    std::vector<dwf_ctx *> members;
    dwf::CoopGate *gate = nullptr;  // owned by the batch context, shared by its members
    std::vector<cudaEvent_t> batch_ev;  // batch context: one join event per member, then the fork event
    bool own_stream = false;        // member streams are created and destroyed by the library
    long long applies64 = 0, applies32 = 0;
    // event profiler
    bool prof = false;
    std::vector<dwf::ProfRecord> prof_rec;
    std::vector<dwf::ProfRecord> *cap_rec = nullptr;  // while a graph is captured: its launches' records
    std::vector<cudaEvent_t> prof_pool;
};

namespace dwf {

// Brackets one kernel launch with profiling events when the profiler is on.
struct ProfScope {
    dwf_ctx *c;
    int cls, units;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(dwf_ctx *ctx, int k, int nunits = 1);
    ~ProfScope();
};
void prof_reset(dwf_ctx *c);
unsigned long long launch_count();

// ---- pack.cu ----
void pack(dwf_ctx *c, void *internal, const double2 *canonical, dwf_prec prec, int nrhs);
void unpack(dwf_ctx *c, double2 *canonical, const void *internal, dwf_prec prec, int nrhs);
void pack_links(dwf_ctx *c, const double2 *U);  // fills U32 from U64

// ---- dslash.cu ----
// out = D in (or D^+) on nrhs fields, precision by pointer type
void dslash(dwf_ctx *c, double2 *out, const double2 *in, bool dag, int nrhs);
void dslash(dwf_ctx *c, float2 *out, const float2 *in, bool dag, int nrhs);
// FP32 D (or D^+) that also writes |out_r|^2 to the double slot slot + r*stride
// (available when dslash_norm_fused(c))
bool dslash_norm_fused(dwf_ctx *c);
void dslash_norm(dwf_ctx *c, float2 *out, const float2 *in, bool dag, int nrhs, int slot, int stride);
// res = b - D x on nrhs FP32 fields (res distinct from x and b; when dslash_norm_fused(c))
void dslash_residual(dwf_ctx *c, float2 *res, const float2 *x, const float2 *b, int nrhs);
// CGNR's w = D p carried without p: w_out = D z + b w_in for every right-hand
// side r, b = scal[inum + r stride] / scal[iden + r stride], and |w_out|^2 into
// scal[slot + r stride] (when dslash_norm_fused(c))
void dslash_wupdate(dwf_ctx *c, float2 *wout, const float2 *z, const float2 *win, int nrhs, int slot, int stride,
                    int inum, int iden);
// CGNR's normal-equations residual update z_out = z_in - a D^+ w for every
// right-hand side r, a = scal[izz + r stride] / scal[iww + r stride], and
// |z_out|^2 into scal[slot + r stride] (available when dslash_norm_fused(c))
void dslash_zupdate(dwf_ctx *c, float2 *zout, const float2 *w, const float2 *zin, int nrhs, int slot, int stride,
                    int izz, int iww);

// ---- blas.cu ---- (n = number of complex elements; slots index ctx->scal)
template <typename T> void bzero(dwf_ctx *c, T *x, int64_t n);
template <typename TO, typename TI> void bcopy(dwf_ctx *c, TO *out, const TI *in, int64_t n);
// slot[k] (double2 view at double index 2k) = <x, y> = sum conj(x) y
template <typename TX, typename TY> void bdot(dwf_ctx *c, int slot, const TX *x, const TY *y, int64_t n);
// slots slot + 2j, slot + 2j + 1 = <V_j, w> for j < k (w read once per 8 vectors)
template <typename T> void bmultidot(dwf_ctx *c, int slot, T *const *V, int k, const T *w, int64_t n);
// slot (double at index k) = |x|^2
template <typename T> void bnorm2(dwf_ctx *c, int slot, const T *x, int64_t n);
double read_scalar(dwf_ctx *c, int dslot);  // synchronises the stream
void read_scalars(dwf_ctx *c, int dslot, int count, double *out);
void write_scalar(dwf_ctx *c, int dslot, double v);

}  // namespace dwf
