// The coarsest-level solve S2 of the V-cycle (Sec. 2: S2 acts on R A P) for
// a batch of right-hand sides, with the coarse stencil on the tensor cores.
//
// With nb right-hand sides the 9-point stencil at one coarse site is a dense
// contraction: y[a][n] = sum_{d, c} Y_d[a][c] x_d[c][n], d over the site and
// its 8 neighbours, a, c over the Nvec components, n over the right-hand
// sides.  In real arithmetic, with A' = [Re Y_d | Im Y_d] (Nvec x 2 Nvec per
// direction) and B' = [[Re x, Im x]; [-Im x, Re x]] (2 Nvec x 2 nb per
// direction), the columns of A' B' are [Re y | Im y].  One site is one MMA
// chain of K = 18 Nvec (kind::f16, BF16 operands, FP32 accumulation in
// tensor memory): A' is the BF16 coarse stencil itself, laid out once per
// setup as a per-site image in the tensor cores' K-major shared-memory
// layout and brought in per site by a bulk copy; B' is built by the threads
// from the FP32 vectors, each value split into a BF16 high part and a BF16
// remainder (two column blocks of B'), so that the product is that of the
// BF16 links with the FP32 vectors up to a relative 2^-16.  Two sites are in
// flight: the copy and the B' build of one overlap the MMAs of the other and
// the read-back of the one before.
//
// The GCR around it is that of the SIMT batched solver (coarse_gcr_batch.cu)
// with one change, the second classical Gram-Schmidt pass runs only where
// the first removed 3/4 or more of |w|^2: |w| normalisation,
// x += <w,r> z, r -= <w,r> w, true residual at each restart, right-hand
// sides leaving the lockstep as they converge.  Element arithmetic, the
// in-warp sums and the per-CTA partials are FP32; every CTA adds all CTAs'
// partials in the same fixed order, so all take identical decisions.  Waits on the copy and the
// MMA completion are bounded (about one second); on expiry the kernel sets
// an error word, every CTA leaves the iteration at the next reduction, and
// the caller reports DWF_ETIMEOUT.
#include <cooperative_groups.h>

#include <cstdio>
#include <cstdlib>
#include <atomic>
#include <cstring>
#include <type_traits>
#include <vector>

#include "mg.cuh"

namespace cg = cooperative_groups;

namespace dwf {

namespace {

constexpr int TCT = 256;                   // threads per CTA
constexpr int TMAXR = 16;                  // restart length
constexpr int TMAXB = 16;                  // right-hand sides per launch
constexpr int TMAXV = (TMAXR + 2) * TMAXB; // complex values reduced per phase
constexpr int TMEM_COLS = 128;             // two stages of at most 64 FP32 columns
constexpr int STAGE_COLS = 64;
constexpr int NWARP = TCT / 32;

// Geometry of one site's operands for Nvec = NV.
template <int NV> struct TcGeom {
    static constexpr int RG = NV / 8;                 // 8-row groups of A'
    static constexpr int KTOT = 18 * NV;              // contraction length
    static constexpr int KC = KTOT / 8;               // 16-byte K chunks
    static constexpr int NMMA = KTOT / 16;            // MMAs per site
    static constexpr int LBO_A = RG * 128;            // byte stride between K chunks of A'
    static constexpr int AIMG = KC * RG * 128;        // bytes of one site's A' image
    // an M = 128 MMA reads 16 row groups from each K chunk: the rows past the
    // site's own (their products are discarded) run into the next chunks, and
    // past the last one into this tail
    static constexpr int ABUF = ((KC - 1) * RG * 128 + 2048 + 1023) / 1024 * 1024;
    static constexpr int SBO_B = KC * 128;            // byte stride between 8-row groups of B'
    static int bbuf(int N) { return ((N / 8) * KC * 128 + 1023) / 1024 * 1024; }
};

struct TcArgs {
    const unsigned char *Aimg;  // [V][AIMG] BF16 A' images
    const int *nbr;             // neighbour table [V][8]
    int V;
    const float2 *b;            // [nb][Nf]
    float2 *x, *r;              // [nb][Nf]
    float2 *Z, *W;              // [restart][nb][Nf]
    float2 *part;               // [2][TMAXV][gridDim.x rounded up to even] per-CTA partial sums, two alternating buffers
    int *err;                   // set on an expired wait
    int *iters;
    double tol;
    int maxiter, restart, nb, nbp;  // nbp: nb rounded up to a multiple of 4
    int bbuf;                   // bytes of one B' stage
    int force_wait;             // test hook: thread 0 of every CTA first waits on a barrier nothing completes
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle, core matrices of
// 8 rows x 16 bytes; lbo = byte stride between core matrices along K,
// sbo = byte stride between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the fifth-generation tensor cores
    return d;
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the given phase of an mbarrier for at most about one second.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    const uint64_t t0 = globaltimer();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
        if (globaltimer() - t0 > 1000000000ull) return false;
    }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Sum over the 32 lanes of P values (P a power of two, P <= 32) in
// 31 - (32 - P) + (5 - log2 P) shuffles: halves of the value set are
// exchanged between lane pairs (a reduce-scatter), then the remaining lane
// bits are summed.  On return lane l holds the total of value
// l >> (5 - log2 P).
template <int P> __device__ __forceinline__ float warp_scatter_sum(float *v) {
    const int lane = threadIdx.x & 31;
    int o = 16;
#pragma unroll
    for (int h = P / 2; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    float s = v[0];
    for (; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}
template <int P> __host__ __device__ constexpr int log2p() { return P <= 1 ? 0 : 1 + log2p<P / 2>(); }

// Per-kernel state of the two-stage pipeline.
struct Pipe {
    uint32_t tmem;          // TMEM base address of the CTA's allocation
    uint32_t phA, phM;      // expected phase bit of each stage's copy / MMA barrier
    uint32_t barA[2], barM[2];
    unsigned char *sA[2], *sB[2];
};

// Read the MMA result of one site back from tensor memory (warp 0) and
// store y = A x for the active right-hand sides.
template <int NV>
__device__ void tc_epilogue(const TcArgs &a, Pipe &pp, int st, int site, float2 *out, const int *act, int Nf,
                            int *bad) {
    const int lane = threadIdx.x & 31;
    if (!mbar_wait(pp.barM[st], (pp.phM >> st) & 1u)) *bad = 1;
    tc_fence_after();
    const int N = 4 * a.nbp;
    float D[STAGE_COLS];
#pragma unroll
    for (int q = 0; q < STAGE_COLS / 16; ++q)
        if (q * 16 < N) tmem_ld16(pp.tmem + (uint32_t)(st * STAGE_COLS + q * 16), D + q * 16);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (lane < NV) {
        // columns [Re hi | Im hi | Re lo | Im lo], nbp each; the lane is row a of the site
        const int nbp = a.nbp;
        for (int n = 0; n < a.nb; ++n)
            if (act[n])
                out[(size_t)n * Nf + (size_t)site * NV + lane] =
                    make_float2(D[n] + D[2 * nbp + n], D[nbp + n] + D[3 * nbp + n]);
    }
}

// out = A in on the CTA's sites [s0, s1) for the active right-hand sides.
template <int NV>
__device__ void tc_apply(const TcArgs &a, Pipe &pp, float2 *out, const float2 *in, int s0, int s1, const int *act,
                         int Nf, int *bad) {
    using Gm = TcGeom<NV>;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nbp = a.nbp, N = 4 * nbp;
    const uint32_t idesc = (1u << 4)                       // D: FP32
                           | (1u << 7) | (1u << 10)        // A, B: BF16
                           | ((uint32_t)(N >> 3) << 17)    // N
                           | ((uint32_t)(128 >> 4) << 24); // M = 128 (rows past Nvec discarded)
    const int nsite = s1 - s0;
    for (int j = 0; j < nsite; ++j) {
        const int s = s0 + j, st = j & 1;
        if (tid == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(pp.barA[st]), "r"(Gm::AIMG)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_addr(pp.sA[st])),
                "l"(a.Aimg + (size_t)s * Gm::AIMG), "r"(Gm::AIMG), "r"(pp.barA[st])
                : "memory");
        }
        // B' of site s: items (direction d, component octet c8, right-hand side n)
        unsigned char *sB = pp.sB[st];
        const int nitem = 9 * (NV / 8) * nbp;
        for (int it = tid; it < nitem; it += TCT) {
            const int n = it % nbp, rest = it / nbp;
            const int c8 = rest % (NV / 8), d = rest / (NV / 8);
            const int sd = d == 0 ? s : a.nbr[s * 8 + d - 1];
            float4 v[4];
            if (n < a.nb && act[n]) {
                const float4 *p = reinterpret_cast<const float4 *>(in + (size_t)n * Nf + (size_t)sd * NV + 8 * c8);
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = __ldcg(p + q);  // neighbours' values come from other CTAs
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            // hi / lo BF16 parts of the 8 real and 8 imaginary parts
            __align__(16) __nv_bfloat16 rh[8], ih[8], rl[8], il[8], nih[8], nil[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float xr0 = v[q].x, xi0 = v[q].y, xr1 = v[q].z, xi1 = v[q].w;
                const __nv_bfloat16 a0 = __float2bfloat16_rn(xr0), b0 = __float2bfloat16_rn(xi0);
                const __nv_bfloat16 a1 = __float2bfloat16_rn(xr1), b1 = __float2bfloat16_rn(xi1);
                rh[2 * q] = a0; ih[2 * q] = b0; rh[2 * q + 1] = a1; ih[2 * q + 1] = b1;
                rl[2 * q] = __float2bfloat16_rn(xr0 - __bfloat162float(a0));
                il[2 * q] = __float2bfloat16_rn(xi0 - __bfloat162float(b0));
                rl[2 * q + 1] = __float2bfloat16_rn(xr1 - __bfloat162float(a1));
                il[2 * q + 1] = __float2bfloat16_rn(xi1 - __bfloat162float(b1));
                nih[2 * q] = __hneg(ih[2 * q]); nih[2 * q + 1] = __hneg(ih[2 * q + 1]);
                nil[2 * q] = __hneg(il[2 * q]); nil[2 * q + 1] = __hneg(il[2 * q + 1]);
            }
            const int kc1 = d * (2 * NV / 8) + c8, kc2 = kc1 + NV / 8;  // Re Y and Im Y columns of A'
            auto row = [&](int q, int kc) -> uint4 * {
                return reinterpret_cast<uint4 *>(sB + (q >> 3) * Gm::SBO_B + kc * 128 + (q & 7) * 16);
            };
            const uint4 RH = *reinterpret_cast<const uint4 *>(rh), IH = *reinterpret_cast<const uint4 *>(ih);
            const uint4 RL = *reinterpret_cast<const uint4 *>(rl), IL = *reinterpret_cast<const uint4 *>(il);
            const uint4 NIH = *reinterpret_cast<const uint4 *>(nih), NIL = *reinterpret_cast<const uint4 *>(nil);
            *row(n, kc1) = RH;               *row(n, kc2) = NIH;
            *row(nbp + n, kc1) = IH;         *row(nbp + n, kc2) = RH;
            *row(2 * nbp + n, kc1) = RL;     *row(2 * nbp + n, kc2) = NIL;
            *row(3 * nbp + n, kc1) = IL;     *row(3 * nbp + n, kc2) = RL;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            const bool ok = mbar_wait(pp.barA[st], (pp.phA >> st) & 1u);
            if (!ok) *bad = 1;
            tc_fence_after();
            if (ok) {
                const uint32_t aa = smem_addr(pp.sA[st]), bb = smem_addr(pp.sB[st]);
                const uint32_t dt = pp.tmem + (uint32_t)(st * STAGE_COLS);
#pragma unroll 1
                for (int kk = 0; kk < Gm::NMMA; ++kk) {
                    const uint64_t da = smem_desc(aa + kk * 2 * Gm::LBO_A, Gm::LBO_A, 128);
                    const uint64_t db = smem_desc(bb + kk * 2 * 128, 128, Gm::SBO_B);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
                        "l"(da), "l"(db), "r"(idesc), "r"(kk)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             pp.barM[st])
                         : "memory");
        }
        pp.phA ^= 1u << st;
        if (warp == 0 && j >= 1) {
            tc_epilogue<NV>(a, pp, st ^ 1, s - 1, out, act, Nf, bad);
            pp.phM ^= 1u << (st ^ 1);
        } else if (j >= 1) {
            pp.phM ^= 1u << (st ^ 1);
        }
        tc_fence_before();
        __syncthreads();
    }
    if (nsite >= 1) {
        const int st = (nsite - 1) & 1;
        if (warp == 0) tc_epilogue<NV>(a, pp, st, s1 - 1, out, act, Nf, bad);
        pp.phM ^= 1u << st;
    }
    tc_fence_before();
    __syncthreads();
}

template <int NV>
__global__ void __launch_bounds__(TCT, 1) coarse_gcr_tc_kernel(TcArgs a) {
    using Gm = TcGeom<NV>;
    cg::grid_group grid = cg::this_grid();
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ float red[NWARP][2 * TMAXV];
    __shared__ double2 tot[TMAXV];
    __shared__ double rn2[TMAXB], stop[TMAXB], wwv[TMAXB];
    __shared__ int act[TMAXB], its[TMAXB];
    __shared__ __align__(8) uint64_t bars[5];  // copy and MMA barriers of the two stages; [4]: the test hook's
    __shared__ uint32_t tbase;
    __shared__ int bad, quit, second;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nb = a.nb, nblk = gridDim.x;
    const int V = a.V, Nf = V * NV;
    const int sites = (V + nblk - 1) / nblk;
    const int s0 = min((int)blockIdx.x * sites, V), s1 = min(s0 + sites, V);
    const int e0 = s0 * NV, E = (s1 - s0) * NV;
    const int Epad = (E + 31) / 32 * 32, nitems = nb * Epad;

    Pipe pp;
    pp.sA[0] = dsm;
    pp.sA[1] = dsm + Gm::ABUF;
    pp.sB[0] = dsm + 2 * Gm::ABUF;
    pp.sB[1] = dsm + 2 * Gm::ABUF + a.bbuf;
    for (int i = 0; i < 2; ++i) {
        pp.barA[i] = smem_addr(&bars[i]);
        pp.barM[i] = smem_addr(&bars[2 + i]);
    }
    pp.phA = pp.phM = 0;
    // the A' tails past the images are read by the discarded rows: keep them finite
    for (int i = tid; i < (Gm::ABUF - Gm::AIMG) / 4; i += TCT) {
        reinterpret_cast<float *>(pp.sA[0] + Gm::AIMG)[i] = 0.f;
        reinterpret_cast<float *>(pp.sA[1] + Gm::AIMG)[i] = 0.f;
    }
    if (tid == 0) {
        for (int i = 0; i < 5; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[i])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        bad = 0;
        quit = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tbase)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    pp.tmem = tbase;
    // A wait that runs out takes the same exit as an expired copy or MMA
    // wait: the flag reaches every CTA through the next reduction, all stop
    // together with x as it stands, and the host reports DWF_ETIMEOUT.
    if (a.force_wait && tid == 0 && !mbar_wait(smem_addr(&bars[4]), 0u)) bad = 1;

    auto zero_red = [&](int nv) {
        for (int q = tid; q < NWARP * 2 * nv; q += TCT) red[q / (2 * nv)][q % (2 * nv)] = 0.f;
        __syncthreads();
    };
    // Totals of the complex values 0..nv-1 into tot[] of every CTA through one
    // grid barrier: each CTA writes its FP32 partials (warps summed in a fixed
    // order) and its error flag to one of two alternating buffers, then every
    // CTA adds all CTAs' partials in the same order, so all hold identical
    // totals and take identical decisions.  The two buffers keep a CTA that
    // runs ahead to the next reduction off the partials others still read.
    // Partials are stored value-major with an even row stride, so a thread
    // reads its value's partials two CTAs at a time in 16-byte loads, many in
    // flight, and still adds them in CTA order.
    int phase = 0;
    const int pstride = (nblk + 1) & ~1;
    auto finish = [&](int nv) {
        __syncthreads();
        float2 *pb = a.part + (size_t)(phase & 1) * TMAXV * pstride;
        for (int p = tid; p <= nv; p += TCT) {
            float2 v = make_float2(0.f, 0.f);
            if (p < nv) {
                for (int w = 0; w < NWARP; ++w) {
                    v.x += red[w][2 * p];
                    v.y += red[w][2 * p + 1];
                }
            } else {
                v.x = bad ? 1.f : 0.f;
            }
            pb[(size_t)p * pstride + blockIdx.x] = v;
        }
        if (tid == 0 && bad) atomicOr(a.err, 1);
        __threadfence();
        grid.sync();
        for (int p = tid; p <= nv; p += TCT) {
            const float4 *row = reinterpret_cast<const float4 *>(pb + (size_t)p * pstride);
            float sx = 0.f, sy = 0.f;
#pragma unroll 16
            for (int q = 0; q < pstride / 2; ++q) {
                const float4 w = __ldcg(row + q);
                sx += w.x;
                sy += w.y;
                if (2 * q + 1 < nblk) {
                    sx += w.z;
                    sy += w.w;
                }
            }
            if (p < nv) tot[p] = make_double2(sx, sy);
            else quit = sx > 0.f;
        }
        ++phase;
        __syncthreads();
    };

    // x = 0, r = b, |b|^2 per right-hand side
    zero_red(nb);
    for (int base = warp * 32; base < nitems; base += TCT) {
        const int rr = base / Epad;
        const int eo = base - rr * Epad + lane;
        float v = 0.f;
        if (eo < E) {
            const int i = rr * Nf + e0 + eo;
            a.x[i] = make_float2(0.f, 0.f);
            const float2 bv = a.b[i];
            a.r[i] = bv;
            v = bv.x * bv.x + bv.y * bv.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][2 * rr] += v;
    }
    finish(nb);
    if (tid < nb) {
        rn2[tid] = tot[tid].x;
        stop[tid] = a.tol * a.tol * tot[tid].x;
        act[tid] = (tot[tid].x > 0.0 && a.maxiter > 0 && !quit) ? 1 : 0;
        its[tid] = 0;
    }
    __syncthreads();

    // Gram-Schmidt dots <W_i, W_k> of the k stored directions (values i*nb + rr);
    // with NORMS also |W_k|^2 (value k*nb + rr) and <W_k, r> ((k+1)*nb + rr)
    auto gs_dots = [&](auto Pc, int k, bool norms) {
        constexpr int P = decltype(Pc)::value;
        constexpr int lp = log2p<P>();
        const float2 *Wk = a.W + (size_t)k * nb * Nf;
        for (int base = warp * 32; base < nitems; base += TCT) {
            const int rr = base / Epad;
            if (!act[rr]) continue;
            const int eo = base - rr * Epad + lane;
            const bool ok = eo < E;
            const int ie = rr * Nf + e0 + eo;
            const float2 w = ok ? Wk[ie] : make_float2(0.f, 0.f);
            if (k > 0) {
                float v[P];
#pragma unroll
                for (int i = 0; i < P / 2; ++i) {
                    float2 u = make_float2(0.f, 0.f);
                    if (i < k && ok) u = a.W[(size_t)i * nb * Nf + ie];
                    v[2 * i] = u.x * w.x + u.y * w.y;
                    v[2 * i + 1] = u.x * w.y - u.y * w.x;
                }
                const float sv = warp_scatter_sum<P>(v);
                const int vi = lane >> (5 - lp);
                if ((lane & ((1 << (5 - lp)) - 1)) == 0 && vi < 2 * k)
                    red[warp][2 * ((vi >> 1) * nb + rr) + (vi & 1)] += sv;
            }
            if (norms) {
                const float2 q = ok ? a.r[ie] : make_float2(0.f, 0.f);
                float u[4] = {w.x * w.x + w.y * w.y, 0.f, w.x * q.x + w.y * q.y, w.x * q.y - w.y * q.x};
                const float su = warp_scatter_sum<4>(u);
                const int ui = lane >> 3;
                if ((lane & 7) == 0) {
                    if (ui == 0) red[warp][2 * (k * nb + rr)] += su;
                    else if (ui >= 2) red[warp][2 * ((k + 1) * nb + rr) + (ui - 2)] += su;
                }
            }
        }
    };
    auto dots = [&](int k, bool norms) {
        if (k <= 1) gs_dots(std::integral_constant<int, 2>{}, k, norms);
        else if (k <= 2) gs_dots(std::integral_constant<int, 4>{}, k, norms);
        else if (k <= 4) gs_dots(std::integral_constant<int, 8>{}, k, norms);
        else if (k <= 8) gs_dots(std::integral_constant<int, 16>{}, k, norms);
        else gs_dots(std::integral_constant<int, 32>{}, k, norms);
    };
    // w -= sum_i beta_i W_i, z -= sum_i beta_i Z_i with beta_i = tot[i*nb + rr]
    auto project_out = [&](int k, float2 &w, float2 &z, int rr, int ie) {
#pragma unroll
        for (int i = 0; i < TMAXR; ++i)
            if (i < k) {
                const float br = (float)tot[i * nb + rr].x, bi = (float)tot[i * nb + rr].y;
                const float2 wi = a.W[(size_t)i * nb * Nf + ie], zi = a.Z[(size_t)i * nb * Nf + ie];
                w.x -= br * wi.x - bi * wi.y;
                w.y -= br * wi.y + bi * wi.x;
                z.x -= br * zi.x - bi * zi.y;
                z.y -= br * zi.y + bi * zi.x;
            }
    };

    int k = 0;
    while (!quit) {
        bool any = false;
        for (int rr = 0; rr < nb; ++rr) any |= act[rr] != 0;
        if (!any) break;
        float2 *Zk = a.Z + (size_t)k * nb * Nf, *Wk = a.W + (size_t)k * nb * Nf;
        for (int base = warp * 32; base < nitems; base += TCT) {
            const int rr = base / Epad;
            const int eo = base - rr * Epad + lane;
            if (act[rr] && eo < E) Zk[rr * Nf + e0 + eo] = a.r[rr * Nf + e0 + eo];
        }
        __threadfence();
        grid.sync();
        tc_apply<NV>(a, pp, Wk, Zk, s0, s1, act, Nf, &bad);
        // Classical Gram-Schmidt against the stored W_i, reduced together with
        // |W_k|^2 and <W_k, r>: after the projection |W_k|^2 loses
        // sum |beta_i|^2 (the W_i are orthonormal) and <W_k, r> is unchanged
        // (r is orthogonal to the W_i in GCR).  Where the projection removes
        // 3/4 or more of |W_k|^2 for some right-hand side, that difference
        // has lost too many digits: the projection is applied and a second
        // pass reduced the same way instead.  Every CTA holds the same totals
        // and so takes the same branch.
        zero_red((k + 2) * nb);
        dots(k, true);
        finish((k + 2) * nb);
        if (quit) break;
        if (k > 0) {
            if (tid == 0) {
                bool again = false;
                for (int rr = 0; rr < nb; ++rr) {
                    if (!act[rr]) continue;
                    double removed = 0.0;
                    for (int i = 0; i < k; ++i)
                        removed += tot[i * nb + rr].x * tot[i * nb + rr].x + tot[i * nb + rr].y * tot[i * nb + rr].y;
                    again |= !(removed < 0.75 * tot[k * nb + rr].x);
                }
                second = again;
            }
            __syncthreads();
            if (second) {
                for (int base = warp * 32; base < nitems; base += TCT) {
                    const int rr = base / Epad;
                    const int eo = base - rr * Epad + lane;
                    if (!act[rr] || eo >= E) continue;
                    const int ie = rr * Nf + e0 + eo;
                    float2 w = Wk[ie], z = Zk[ie];
                    project_out(k, w, z, rr, ie);
                    Wk[ie] = w;
                    Zk[ie] = z;
                }
                __syncthreads();
                zero_red((k + 2) * nb);
                dots(k, true);
                finish((k + 2) * nb);
                if (quit) break;
            }
        }
        if (tid < nb) {
            double ww = tot[k * nb + tid].x;
            for (int i = 0; i < k; ++i) ww -= tot[i * nb + tid].x * tot[i * nb + tid].x + tot[i * nb + tid].y * tot[i * nb + tid].y;
            wwv[tid] = ww;
        }
        __syncthreads();
        for (int base = warp * 32; base < nitems; base += TCT) {
            const int rr = base / Epad;
            const int eo = base - rr * Epad + lane;
            if (!act[rr] || eo >= E) continue;
            const double ww = wwv[rr];
            if (!(ww > 0.0)) continue;  // breakdown: handled below, the same in every CTA
            const double inv = 1.0 / sqrt(ww);
            const double2 wr = tot[(k + 1) * nb + rr];
            const float sc = (float)inv, arr = (float)(wr.x * inv), aii = (float)(wr.y * inv);
            const int ie = rr * Nf + e0 + eo;
            float2 z = Zk[ie], w = Wk[ie], xx = a.x[ie], q = a.r[ie];
            project_out(k, w, z, rr, ie);
            z.x *= sc; z.y *= sc; w.x *= sc; w.y *= sc;
            xx.x += arr * z.x - aii * z.y;
            xx.y += arr * z.y + aii * z.x;
            q.x -= arr * w.x - aii * w.y;
            q.y -= arr * w.y + aii * w.x;
            Zk[ie] = z; Wk[ie] = w; a.x[ie] = xx; a.r[ie] = q;
        }
        __syncthreads();
        if (tid < nb && act[tid]) {
            const double ww = wwv[tid];
            if (!(ww > 0.0)) {
                act[tid] = 0;
            } else {
                const double2 wr = tot[(k + 1) * nb + tid];
                rn2[tid] -= (wr.x * wr.x + wr.y * wr.y) / ww;
                its[tid]++;
                if (rn2[tid] <= stop[tid] || its[tid] >= a.maxiter) act[tid] = 0;
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
                tc_apply<NV>(a, pp, a.r, a.x, s0, s1, act, Nf, &bad);
                zero_red(nb);
                for (int base = warp * 32; base < nitems; base += TCT) {
                    const int rr = base / Epad;
                    if (!act[rr]) continue;
                    const int eo = base - rr * Epad + lane;
                    float v = 0.f;
                    if (eo < E) {
                        const int ie = rr * Nf + e0 + eo;
                        const float2 bv = a.b[ie], ax = a.r[ie];
                        const float2 q = make_float2(bv.x - ax.x, bv.y - ax.y);
                        a.r[ie] = q;
                        v = q.x * q.x + q.y * q.y;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) red[warp][2 * rr] += v;
                }
                finish(nb);
                if (quit) break;
                if (tid < nb && act[tid]) {
                    rn2[tid] = tot[tid].x;
                    if (rn2[tid] <= stop[tid]) act[tid] = 0;
                }
                __syncthreads();
            }
            k = 0;
        }
    }
    if (blockIdx.x == 0 && tid == 0) {
        int s = 0;
        for (int rr = 0; rr < nb; ++rr) s += its[rr];
        atomicAdd(a.iters, s);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(pp.tmem), "r"(TMEM_COLS));
}

// A' images of the BF16 coarse stencil, one per site: element (a, k) with
// k = 2 Nvec d + c (Re Y_d[a][c]) or 2 Nvec d + Nvec + c (Im Y_d[a][c]) at
// byte (k / 8) LBO_A + (a / 8) 128 + (a % 8) 16 + (k % 8) 2.  The values are
// rounded FP64 -> FP32 -> BF16 as in the library's BF16 stencil copy.
template <int NV>
__global__ void tc_image_kernel(__nv_bfloat16 *__restrict__ img, const double2 *__restrict__ Y, int64_t V) {
    using Gm = TcGeom<NV>;
    const int64_t n = V * 9 * NV * NV;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % NV);
        const int aa = (int)((i / NV) % NV);
        const int d = (int)((i / (NV * NV)) % 9);
        const int64_t site = i / (9 * NV * NV);
        const double2 y = Y[i];  // Y[site][d][a][c]
        unsigned char *base = reinterpret_cast<unsigned char *>(img) + site * Gm::AIMG;
        const int k1 = 2 * NV * d + c, k2 = k1 + NV;
        const int roff = (aa >> 3) * 128 + (aa & 7) * 16;
        *reinterpret_cast<__nv_bfloat16 *>(base + (k1 >> 3) * Gm::LBO_A + roff + (k1 & 7) * 2) =
            __float2bfloat16_rn((float)y.x);
        *reinterpret_cast<__nv_bfloat16 *>(base + (k2 >> 3) * Gm::LBO_A + roff + (k2 & 7) * 2) =
            __float2bfloat16_rn((float)y.y);
    }
}

template <int NV> size_t tc_smem(int nb) {
    using Gm = TcGeom<NV>;
    const int nbp = (nb + 3) / 4 * 4;
    return 2 * (size_t)Gm::ABUF + 2 * (size_t)Gm::bbuf(4 * nbp);
}

template <int NV> void *tc_kernel_fn() { return (void *)coarse_gcr_tc_kernel<NV>; }

size_t tc_static_smem() {
    return sizeof(float) * NWARP * 2 * TMAXV + sizeof(double2) * TMAXV + 2 * sizeof(double) * TMAXB +
           2 * sizeof(int) * TMAXB + 5 * sizeof(uint64_t) + 4 * sizeof(int) + 64;
}

template <int NV> bool tc_fits(dwf_ctx *c, int nb) {
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return tc_smem<NV>(nb) + tc_static_smem() <= (size_t)optin;
}

bool tc_shape_ok(dwf_ctx *c, const Level &L, int nb) {
    if (L.yprec != DWF_BF16 || L.npts != 9 || nb < 1 || nb > TMAXB) return false;
    switch (L.lg.ncomp) {
        case 8: return tc_fits<8>(c, nb);
        case 16: return tc_fits<16>(c, nb);
        case 24: return tc_fits<24>(c, nb);
        case 32: return tc_fits<32>(c, nb);
        default: return false;
    }
}

// Test hook for the bounded waits: DWF_TC_FORCE_WAIT=n in the environment
// makes the first n solver launches outside stream capture start with a wait
// that nothing completes, so that it runs out (after about one second).
bool forced_wait(dwf_ctx *c) {
    static std::atomic<int> left{[] {
        const char *e = getenv("DWF_TC_FORCE_WAIT");
        return e ? std::max(0, atoi(e)) : 0;
    }()};
    if (left.load() <= 0) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    DWF_CUDA(cudaStreamIsCapturing(c->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone) return false;
    return left.fetch_sub(1) > 0;
}

template <int NV>
void launch_tc(dwf_ctx *c, const Level &L, float2 *x, const float2 *b, int nb, float2 *r, float2 *Z, float2 *W,
               double2 *part, int *iters, double tol, int maxiter, int restart) {
    TcArgs a;
    a.Aimg = L.Ytc.as<unsigned char>();
    a.nbr = L.nbr.as<int>();
    a.V = (int)L.lg.g.V;
    a.b = b;
    a.x = x;
    a.r = r;
    a.Z = Z;
    a.W = W;
    // two alternating buffers of FP32 partials: as many bytes as the caller's FP64 partials and totals
    static_assert(2 * sizeof(float2) == sizeof(double2), "partial-sum buffer size");
    a.part = reinterpret_cast<float2 *>(part);
    if (!c->tc_err.p) {
        c->tc_err.alloc(sizeof(int));
        DWF_CUDA(cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream));
    }
    a.err = c->tc_err.as<int>();
    a.iters = iters;
    a.tol = tol;
    a.maxiter = maxiter;
    a.restart = restart;
    a.nb = nb;
    a.nbp = (nb + 3) / 4 * 4;
    a.bbuf = TcGeom<NV>::bbuf(4 * a.nbp);
    a.force_wait = 0;
    c->tc_used = true;
    void *kargs[] = {&a};
    void *fn = tc_kernel_fn<NV>();
    const size_t smem = tc_smem<NV>(nb);
    DWF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    DWF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TCT, smem));
    DWF_REQUIRE(per_sm >= 1, DWF_ECUDA, "tensor-core coarse solver cannot be co-resident");
    // The grid (sites per CTA) is the solver's tile: fewer CTAs make the grid
    // barriers cheaper and the per-CTA stencil pipeline longer.  The first
    // solve of a shape (coarse sites, Nvec, batch width) in a context times
    // the co-resident candidates of 2, 4, 8, ... sites per CTA on its own
    // inputs (every trial starts from x = 0, so they are repeatable; one
    // untimed run first warms the caches), stopping once a candidate is 30%
    // slower than the best, and keeps the fastest for that shape; the solve
    // itself then runs with it.
    const int64_t V = L.lg.g.V, maxg = (int64_t)per_sm * c->sm_count;
    int nblk = 0;
    for (const auto &e : c->tc_grid)
        if (e[0] == V && e[1] == NV && e[2] == nb) nblk = (int)e[3];
    if (nblk == 0) {
        std::vector<int> cand;
        for (int64_t s = 2; s <= 64; s *= 2) {
            const int64_t g = (V + s - 1) / s;
            if (g <= maxg && g <= c->sm_count && (cand.empty() || cand.back() != (int)g)) cand.push_back((int)g);
            if (g == 1) break;
        }
        if (cand.empty()) cand.push_back((int)std::max<int64_t>(1, std::min<int64_t>(V, c->sm_count)));
        nblk = cand[0];
        if (cand.size() > 1) {
            if (!c->tc_trial.p) c->tc_trial.alloc(sizeof(int));
            TcArgs t = a;
            t.iters = c->tc_trial.as<int>();
            void *targs[] = {&t};
            cudaEvent_t e0, e1;
            DWF_CUDA(cudaEventCreate(&e0));
            DWF_CUDA(cudaEventCreate(&e1));
            DWF_CUDA(coop_launch(c, fn, dim3((unsigned)cand[0]), dim3(TCT), targs, smem));
            DWF_CHECK_LAUNCH();
            float best = 1e30f;
            for (int g : cand) {
                DWF_CUDA(cudaEventRecord(e0, c->stream));
                DWF_CUDA(coop_launch(c, fn, dim3((unsigned)g), dim3(TCT), targs, smem));
                DWF_CHECK_LAUNCH();
                DWF_CUDA(cudaEventRecord(e1, c->stream));
                DWF_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                DWF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (const char *v = getenv("DWF_VERBOSE"); v && atoi(v) > 0)
                    fprintf(stderr, "[dwfmg] tensor-core coarse solve, %d right-hand sides: %d CTAs %.3f ms\n", nb, g,
                            ms);
                if (ms < best) {
                    best = ms;
                    nblk = g;
                } else if (ms > 1.3f * best) {
                    break;  // fewer CTAs only get slower from here
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
        c->tc_grid.push_back({V, (int64_t)NV, (int64_t)nb, (int64_t)nblk});
    }
    a.force_wait = forced_wait(c) ? 1 : 0;
    DWF_CUDA(coop_launch(c, fn, dim3((unsigned)nblk), dim3(TCT), kargs, smem));
    DWF_CHECK_LAUNCH();
}

}  // namespace

bool coarse_gcr_tc_ok(dwf_ctx *c, const Level &L, int restart, int nb) {
    return restart >= 1 && restart <= TMAXR && L.Ytc.p && tc_shape_ok(c, L, nb);
}

void coarse_gcr_tc(dwf_ctx *c, const Level &L, float2 *x, const float2 *b, int nb, float2 *r, float2 *Z, float2 *W,
                   double2 *part, int *iters, double tol, int maxiter, int restart) {
    DWF_REQUIRE(coarse_gcr_tc_ok(c, L, restart, nb), DWF_EINVAL, "tensor-core coarse solve: unsupported shape");
    ProfScope ps(c, K_COARSE, nb);
    switch (L.lg.ncomp) {
        case 8: launch_tc<8>(c, L, x, b, nb, r, Z, W, part, iters, tol, maxiter, restart); break;
        case 16: launch_tc<16>(c, L, x, b, nb, r, Z, W, part, iters, tol, maxiter, restart); break;
        case 24: launch_tc<24>(c, L, x, b, nb, r, Z, W, part, iters, tol, maxiter, restart); break;
        case 32: launch_tc<32>(c, L, x, b, nb, r, Z, W, part, iters, tol, maxiter, restart); break;
    }
}

void check_tc_timeout(dwf_ctx *c) {
    if (!c->tc_used) return;
    c->tc_used = false;
    DWF_CUDA(cudaMemcpyAsync(c->hscal, c->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    DWF_CUDA(cudaStreamSynchronize(c->stream));
    int e = 0;
    std::memcpy(&e, c->hscal, sizeof(int));
    if (e != 0) DWF_CUDA(cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream));
    DWF_REQUIRE(e == 0, DWF_ETIMEOUT, "tensor-core coarse solve: a bounded wait on the tensor cores expired");
}

// Build the per-site A' images of a level with a BF16 9-point stencil whose
// Nvec the tensor-core solver handles (8, 16, 24, 32); other levels get none.
void build_tc_images(dwf_ctx *c, Level &L) {
    const int n = L.lg.ncomp;
    if (L.yprec != DWF_BF16 || L.npts != 9 || !(n == 8 || n == 16 || n == 24 || n == 32)) {
        L.Ytc.release();
        return;
    }
    const int64_t V = L.lg.g.V;
    const size_t bytes = (size_t)V * 9 * n * n * 4;  // the image holds exactly the BF16 stencil
    if (L.Ytc.bytes < bytes) L.Ytc.alloc(bytes);
    const unsigned blocks = (unsigned)std::min<int64_t>((V * 9 * n * n + 255) / 256, (int64_t)c->sm_count * 16);
    switch (n) {
        case 8: tc_image_kernel<8><<<blocks, 256, 0, c->stream>>>(L.Ytc.as<__nv_bfloat16>(), L.Y64.as<double2>(), V); break;
        case 16: tc_image_kernel<16><<<blocks, 256, 0, c->stream>>>(L.Ytc.as<__nv_bfloat16>(), L.Y64.as<double2>(), V); break;
        case 24: tc_image_kernel<24><<<blocks, 256, 0, c->stream>>>(L.Ytc.as<__nv_bfloat16>(), L.Y64.as<double2>(), V); break;
        case 32: tc_image_kernel<32><<<blocks, 256, 0, c->stream>>>(L.Ytc.as<__nv_bfloat16>(), L.Y64.as<double2>(), V); break;
    }
    DWF_CHECK_LAUNCH();
}

}  // namespace dwf
