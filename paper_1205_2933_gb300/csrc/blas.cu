// Level-1 vector kernels.  Reductions accumulate in FP64 whatever the
// storage precision and are deterministic: every CTA writes a partial sum,
// and the last CTA to finish (atomic ticket) adds the partials in a fixed
// order and stores the result in a device scalar slot, so that solver
// coefficients can stay on the GPU.
#include "dwf_internal.cuh"

namespace dwf {

namespace {

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1024;

__device__ __forceinline__ double2 to_d(double2 a) { return a; }
__device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }

__device__ __forceinline__ double2 block_sum(double2 v, double2 *sh) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : make_double2(0, 0);
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, o);
            v.y += __shfl_down_sync(0xffffffffu, v.y, o);
        }
    __syncthreads();
    return v;  // valid in thread 0
}

// finish: last CTA reduces the partials; writes out[0] (and out[1] for complex)
__device__ void finish(double2 mine, double2 *part, unsigned *count, double *out, bool complex_result) {
    __shared__ double2 sh[32];
    __shared__ bool last;
    double2 t = block_sum(mine, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = t;
        __threadfence();
        unsigned ticket = atomicAdd(count, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double2 v = make_double2(0, 0);
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
        const volatile double *pp = reinterpret_cast<const volatile double *>(&part[i]);
        v.x += pp[0];
        v.y += pp[1];
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0) {
        out[0] = v.x;
        if (complex_result) out[1] = v.y;
        *count = 0u;
    }
}

// Per-thread partial sums in the storage precision (FP32 FMAs for FP32
// fields), combined across threads and CTAs in FP64.
template <typename T> struct Acc;
template <> struct Acc<double2> { using type = double; };
template <> struct Acc<float2> { using type = float; };

template <typename TX, typename TY>
__global__ void __launch_bounds__(RED_THREADS) dot_kernel(const TX *__restrict__ x, const TY *__restrict__ y, int64_t n,
                                                          double2 *part, unsigned *count, double *out) {
    using A = typename Acc<TX>::type;
    A ar = 0, ai = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        TX u = x[i];
        TY v = y[i];
        ar += (A)u.x * (A)v.x + (A)u.y * (A)v.y;
        ai += (A)u.x * (A)v.y - (A)u.y * (A)v.x;
    }
    finish(make_double2((double)ar, (double)ai), part, count, out, true);
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) norm2_kernel(const T *__restrict__ x, int64_t n, double2 *part,
                                                            unsigned *count, double *out) {
    using A = typename Acc<T>::type;
    A a = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T u = x[i];
        a += (A)u.x * (A)u.x + (A)u.y * (A)u.y;
    }
    finish(make_double2((double)a, 0.0), part, count, out, false);
}

// out[2j], out[2j+1] = <V_j, w> for j < K: w is read once for K vectors.
template <typename T, int K> struct MultiDotArgs {
    const T *v[K];
};

template <typename T, int K>
__global__ void __launch_bounds__(RED_THREADS) multidot_kernel(MultiDotArgs<T, K> a, const T *__restrict__ w, int64_t n,
                                                               double2 *part, unsigned *count, double *out) {
    using A = typename Acc<T>::type;
    A ar[K], ai[K];
#pragma unroll
    for (int j = 0; j < K; ++j) ar[j] = ai[j] = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T y = w[i];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            T u = a.v[j][i];
            ar[j] += (A)u.x * (A)y.x + (A)u.y * (A)y.y;
            ai[j] += (A)u.x * (A)y.y - (A)u.y * (A)y.x;
        }
    }
    __shared__ double2 sh[32];
    __shared__ bool last;
    for (int j = 0; j < K; ++j) {
        double2 t = block_sum(make_double2((double)ar[j], (double)ai[j]), sh);
        if (threadIdx.x == 0) part[(size_t)j * gridDim.x + blockIdx.x] = t;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned ticket = atomicAdd(count, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int j = 0; j < K; ++j) {
        double2 v = make_double2(0, 0);
        for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
            const volatile double *pp = reinterpret_cast<const volatile double *>(&part[(size_t)j * gridDim.x + i]);
            v.x += pp[0];
            v.y += pp[1];
        }
        v = block_sum(v, sh);
        if (threadIdx.x == 0) {
            out[2 * j] = v.x;
            out[2 * j + 1] = v.y;
        }
    }
    if (threadIdx.x == 0) *count = 0u;
}

template <typename T>
__global__ void zero_kernel(T *x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = cvt<T, double2>(make_double2(0, 0));
}

template <typename TO, typename TI>
__global__ void copy_kernel(TO *__restrict__ out, const TI *__restrict__ in, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = cvt<TO, TI>(in[i]);
}

unsigned red_blocks(dwf_ctx *c, int64_t n) {
    int64_t b = (n + RED_THREADS - 1) / RED_THREADS;
    int64_t cap = std::min<int64_t>(RED_MAX_BLOCKS, (int64_t)c->sm_count * 6);
    return (unsigned)std::max<int64_t>(1, std::min(b, cap));
}

unsigned ew_blocks(dwf_ctx *c, int64_t n) {
    int64_t b = (n + 255) / 256;
    int64_t cap = (int64_t)c->sm_count * 16;
    return (unsigned)std::max<int64_t>(1, std::min(b, cap));
}

}  // namespace

template <typename T> void bzero(dwf_ctx *c, T *x, int64_t n) {
    zero_kernel<T><<<ew_blocks(c, n), 256, 0, c->stream>>>(x, n);
    DWF_CHECK_LAUNCH();
}

template <typename TO, typename TI> void bcopy(dwf_ctx *c, TO *out, const TI *in, int64_t n) {
    copy_kernel<TO, TI><<<ew_blocks(c, n), 256, 0, c->stream>>>(out, in, n);
    DWF_CHECK_LAUNCH();
}

template <typename TX, typename TY> void bdot(dwf_ctx *c, int slot, const TX *x, const TY *y, int64_t n) {
    dot_kernel<TX, TY><<<red_blocks(c, n), RED_THREADS, 0, c->stream>>>(
        x, y, n, c->red_part.as<double2>(), c->red_count.as<unsigned>(), c->scal.as<double>() + slot);
    DWF_CHECK_LAUNCH();
}

template <typename T> void bnorm2(dwf_ctx *c, int slot, const T *x, int64_t n) {
    norm2_kernel<T><<<red_blocks(c, n), RED_THREADS, 0, c->stream>>>(
        x, n, c->red_part.as<double2>(), c->red_count.as<unsigned>(), c->scal.as<double>() + slot);
    DWF_CHECK_LAUNCH();
}

static unsigned long long g_launches = 0;
void note_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }
void note_launches(unsigned long long n) { __atomic_add_fetch(&g_launches, n, __ATOMIC_RELAXED); }
unsigned long long launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

static cudaEvent_t take_event(dwf_ctx *c) {
    if (!c->prof_pool.empty()) {
        cudaEvent_t e = c->prof_pool.back();
        c->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    DWF_CUDA(cudaEventCreate(&e));
    return e;
}

// Inside a graph capture the events are recorded as event-record nodes of
// the graph (cudaEventRecordExternal), so that every replay records them.
static cudaError_t record(dwf_ctx *c, cudaEvent_t e) {
    return c->cap_rec ? cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal) : cudaEventRecord(e, c->stream);
}

ProfScope::ProfScope(dwf_ctx *ctx, int k, int nunits) : c(ctx), cls(k), units(nunits) {
    if (!c->prof) return;
    a = take_event(c);
    b = take_event(c);
    DWF_CUDA(record(c, a));
}

ProfScope::~ProfScope() {
    if (!a) return;
    if (record(c, b) == cudaSuccess)
        (c->cap_rec ? *c->cap_rec : c->prof_rec).push_back(ProfRecord{cls, a, b, units, -1.f});
}

void prof_reset(dwf_ctx *c) {
    for (auto &r : c->prof_rec)
        if (r.a) {
            c->prof_pool.push_back(r.a);
            c->prof_pool.push_back(r.b);
        }
    c->prof_rec.clear();
}

template <typename T> void bmultidot(dwf_ctx *c, int slot, T *const *V, int k, const T *w, int64_t n) {
    for (int j0 = 0; j0 < k; j0 += 8) {
        int kk = std::min(8, k - j0);
        unsigned nb = red_blocks(c, n);
#define MD(K)                                                                                            \
    {                                                                                                    \
        MultiDotArgs<T, K> a;                                                                            \
        for (int j = 0; j < K; ++j) a.v[j] = V[j0 + j];                                                  \
        multidot_kernel<T, K><<<nb, RED_THREADS, 0, c->stream>>>(a, w, n, c->red_part.as<double2>(),     \
                                                                 c->red_count.as<unsigned>(),            \
                                                                 c->scal.as<double>() + slot + 2 * j0);  \
    }
        switch (kk) {
            case 1: MD(1) break;
            case 2: MD(2) break;
            case 3: MD(3) break;
            case 4: MD(4) break;
            case 5: MD(5) break;
            case 6: MD(6) break;
            case 7: MD(7) break;
            default: MD(8) break;
        }
#undef MD
        DWF_CHECK_LAUNCH();
    }
}

double read_scalar(dwf_ctx *c, int slot) {
    double v;
    read_scalars(c, slot, 1, &v);
    return v;
}

void read_scalars(dwf_ctx *c, int slot, int count, double *out) {
    DWF_CUDA(cudaMemcpyAsync(c->hscal, c->scal.as<double>() + slot, sizeof(double) * count,
                             cudaMemcpyDeviceToHost, c->stream));
    DWF_CUDA(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < count; ++i) out[i] = c->hscal[i];
}

void write_scalar(dwf_ctx *c, int slot, double v) {
    DWF_CUDA(cudaMemcpyAsync(c->scal.as<double>() + slot, &v, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    DWF_CUDA(cudaStreamSynchronize(c->stream));
}

#define INST2(TX, TY) template void bdot<TX, TY>(dwf_ctx *, int, const TX *, const TY *, int64_t); \
                      template void bcopy<TX, TY>(dwf_ctx *, TX *, const TY *, int64_t);
INST2(double2, double2)
INST2(double2, float2)
INST2(float2, double2)
INST2(float2, float2)
template void bzero<double2>(dwf_ctx *, double2 *, int64_t);
template void bzero<float2>(dwf_ctx *, float2 *, int64_t);
template void bnorm2<double2>(dwf_ctx *, int, const double2 *, int64_t);
template void bmultidot<double2>(dwf_ctx *, int, double2 *const *, int, const double2 *, int64_t);
template void bmultidot<float2>(dwf_ctx *, int, float2 *const *, int, const float2 *, int64_t);
template void bnorm2<float2>(dwf_ctx *, int, const float2 *, int64_t);

}  // namespace dwf
