// FP32 fine Dslash with two fifth-dimension slices per thread.
//
// Same operator as dslash.cu (Sec. 2: Shamir domain-wall operator; Sec. 4:
// 11-site stencil).  A thread owns the slices s0 = 2j and s1 = 2j + 1 of one
// 4D site.  Every complex quantity is held as two register pairs: the real
// parts (s0, s1) and the imaginary parts (s0, s1).  The link is the same
// for both slices, so each complex multiply-add of the 3x3 link products is
// four packed FP32x2 FMAs for the two slices (fma.rn.f32x2) instead of eight
// scalar FMAs, and multiplications by +-i are a choice of operands, not
// arithmetic.  Component loads are 16 bytes (the two slices of one
// component are adjacent in the s-fastest layout).  Links are staged once
// per CTA in shared memory, scaled by their hop coefficient and duplicated
// into (re, re, im, im) so that one 16-byte shared load gives both packed
// operands.  The fifth-dimension neighbours come from the thread's own pair
// and from the neighbouring lane (warp shuffles).
#include <algorithm>
#include <cstdint>

#include "dwf_internal.cuh"

namespace dwf {

namespace {

struct P2 {
    unsigned long long v;
};

__device__ __forceinline__ P2 pk(float a, float b) {
    P2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 unpk(P2 p) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(p.v));
    return r;
}
__device__ __forceinline__ P2 fma2(P2 a, P2 b, P2 c) {
    P2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ P2 add2(P2 a, P2 b) {
    P2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ P2 sub2(P2 a, P2 b) {
    P2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ P2 mul2(P2 a, P2 b) {
    P2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

// a complex number for the two slices: real parts and imaginary parts
struct CP {
    P2 re, im;
};

// the half-spinor rows of (1 + sig g_mu) p for both slices; p[k] holds
// component k = spin*3 + colour as (re_s0, im_s0, re_s1, im_s1)
template <int MU>
__device__ __forceinline__ void project2(const float4 p[12], float sig, CP h[6]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float4 p0 = p[a], p1 = p[3 + a], p2 = p[6 + a], p3 = p[9 + a];
        if (MU == 0) {  // h0 = p0 + sig i p3, h1 = p1 + sig i p2
            h[a].re = pk(p0.x - sig * p3.y, p0.z - sig * p3.w);
            h[a].im = pk(p0.y + sig * p3.x, p0.w + sig * p3.z);
            h[3 + a].re = pk(p1.x - sig * p2.y, p1.z - sig * p2.w);
            h[3 + a].im = pk(p1.y + sig * p2.x, p1.w + sig * p2.z);
        } else if (MU == 1) {  // h0 = p0 - sig p3, h1 = p1 + sig p2
            h[a].re = pk(p0.x - sig * p3.x, p0.z - sig * p3.z);
            h[a].im = pk(p0.y - sig * p3.y, p0.w - sig * p3.w);
            h[3 + a].re = pk(p1.x + sig * p2.x, p1.z + sig * p2.z);
            h[3 + a].im = pk(p1.y + sig * p2.y, p1.w + sig * p2.w);
        } else if (MU == 2) {  // h0 = p0 + sig i p2, h1 = p1 - sig i p3
            h[a].re = pk(p0.x - sig * p2.y, p0.z - sig * p2.w);
            h[a].im = pk(p0.y + sig * p2.x, p0.w + sig * p2.z);
            h[3 + a].re = pk(p1.x + sig * p3.y, p1.z + sig * p3.w);
            h[3 + a].im = pk(p1.y - sig * p3.x, p1.w - sig * p3.z);
        } else {  // h0 = p0 + sig p2, h1 = p1 + sig p3
            h[a].re = pk(p0.x + sig * p2.x, p0.z + sig * p2.z);
            h[a].im = pk(p0.y + sig * p2.y, p0.w + sig * p2.w);
            h[3 + a].re = pk(p1.x + sig * p3.x, p1.z + sig * p3.z);
            h[3 + a].im = pk(p1.y + sig * p3.y, p1.w + sig * p3.w);
        }
    }
}

// acc += (1 + sig g_mu) rebuilt from the link products u (rows 0, 1):
//   g_x: row2 = -sig i u1, row3 = -sig i u0     g_y: row2 = sig u1, row3 = -sig u0
//   g_z: row2 = -sig i u0, row3 =  sig i u1     g_t: row2 = sig u0, row3 =  sig u1
// with -i u = (u.im, -u.re) and i u = (-u.im, u.re).
template <int MU>
__device__ __forceinline__ void recon2(CP acc[12], int a, const CP &u0, const CP &u1, float sig) {
    acc[a].re = add2(acc[a].re, u0.re);
    acc[a].im = add2(acc[a].im, u0.im);
    acc[3 + a].re = add2(acc[3 + a].re, u1.re);
    acc[3 + a].im = add2(acc[3 + a].im, u1.im);
    const bool pos = sig > 0.f;
    CP &r2 = acc[6 + a], &r3 = acc[9 + a];
    if (MU == 0) {  // row2 += -sig i u1 = sig (u1.im, -u1.re); row3 += sig (u0.im, -u0.re)
        if (pos) { r2.re = add2(r2.re, u1.im); r2.im = sub2(r2.im, u1.re); r3.re = add2(r3.re, u0.im); r3.im = sub2(r3.im, u0.re); }
        else     { r2.re = sub2(r2.re, u1.im); r2.im = add2(r2.im, u1.re); r3.re = sub2(r3.re, u0.im); r3.im = add2(r3.im, u0.re); }
    } else if (MU == 1) {  // row2 += sig u1; row3 -= sig u0
        if (pos) { r2.re = add2(r2.re, u1.re); r2.im = add2(r2.im, u1.im); r3.re = sub2(r3.re, u0.re); r3.im = sub2(r3.im, u0.im); }
        else     { r2.re = sub2(r2.re, u1.re); r2.im = sub2(r2.im, u1.im); r3.re = add2(r3.re, u0.re); r3.im = add2(r3.im, u0.im); }
    } else if (MU == 2) {  // row2 += sig (u0.im, -u0.re); row3 += sig (-u1.im, u1.re)
        if (pos) { r2.re = add2(r2.re, u0.im); r2.im = sub2(r2.im, u0.re); r3.re = sub2(r3.re, u1.im); r3.im = add2(r3.im, u1.re); }
        else     { r2.re = sub2(r2.re, u0.im); r2.im = add2(r2.im, u0.re); r3.re = add2(r3.re, u1.im); r3.im = sub2(r3.im, u1.re); }
    } else {  // row2 += sig u0; row3 += sig u1
        if (pos) { r2.re = add2(r2.re, u0.re); r2.im = add2(r2.im, u0.im); r3.re = add2(r3.re, u1.re); r3.im = add2(r3.im, u1.im); }
        else     { r2.re = sub2(r2.re, u0.re); r2.im = sub2(r2.im, u0.im); r3.re = sub2(r3.re, u1.re); r3.im = sub2(r3.im, u1.im); }
    }
}

// One 4D hop for both slices from the neighbour's preloaded row p (the 12
// components of the thread's two slices).  sL: the staged link (9 elements
// as float4 (re, re, im, im), hop coefficient included); ADJ: use its
// adjoint.
template <int MU, bool ADJ>
__device__ __forceinline__ void hop2(CP acc[12], const float4 p[12], const float4 *sL, float sig) {
    CP h[6];
    project2<MU>(p, sig, h);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // u[sp] = sum_b M(a,b) h[sp][b]; M = U (a,b) or conj(U (b,a))
        P2 rp0 = pk(0.f, 0.f), rn0 = rp0, ip0 = rp0, in0 = rp0;
        P2 rp1 = rp0, rn1 = rp0, ip1 = rp0, in1 = rp0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float4 m = ADJ ? sL[b * 3 + a] : sL[a * 3 + b];
            const P2 mre = pk(m.x, m.y), mim = pk(m.z, m.w);
            const CP &h0 = h[b], &h1 = h[3 + b];
            if (!ADJ) {  // (mre + i mim)(h.re + i h.im)
                rp0 = fma2(mre, h0.re, rp0); rn0 = fma2(mim, h0.im, rn0);
                ip0 = fma2(mre, h0.im, ip0); ip0 = fma2(mim, h0.re, ip0);
                rp1 = fma2(mre, h1.re, rp1); rn1 = fma2(mim, h1.im, rn1);
                ip1 = fma2(mre, h1.im, ip1); ip1 = fma2(mim, h1.re, ip1);
            } else {     // (mre - i mim)(h.re + i h.im)
                rp0 = fma2(mre, h0.re, rp0); rp0 = fma2(mim, h0.im, rp0);
                ip0 = fma2(mre, h0.im, ip0); in0 = fma2(mim, h0.re, in0);
                rp1 = fma2(mre, h1.re, rp1); rp1 = fma2(mim, h1.im, rp1);
                ip1 = fma2(mre, h1.im, ip1); in1 = fma2(mim, h1.re, in1);
            }
        }
        CP u0, u1;
        if (!ADJ) {
            u0.re = sub2(rp0, rn0); u0.im = ip0;
            u1.re = sub2(rp1, rn1); u1.im = ip1;
        } else {
            u0.re = rp0; u0.im = sub2(ip0, in0);
            u1.re = rp1; u1.im = sub2(ip1, in1);
        }
        recon2<MU>(acc, a, u0, u1, sig);
    }
}

// the 12 components of a thread's two slices in one site's row
template <int LS> __device__ __forceinline__ void ldrow(float4 p[12], const float2 *__restrict__ row) {
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = *reinterpret_cast<const float4 *>(row + k * LS);
}

// CTA = spb whole 4D sites x LS/2 threads; LS/2 divides 32 so that the
// threads of a site share a warp.  A site's 72 staged link elements are
// LSTRIDE = 73 float4 apart: the sites of one warp then start 4 banks apart
// and their broadcast reads of the same element need one shared-memory
// wavefront instead of one per site.
constexpr int LSTRIDE = 73;

// The normal-equations residual update of CGNR, z <- z - a D^+ w, with
// a = zz / ww of each right-hand side read from the scalar slots.
struct ZUpdate {
    const float2 *zin;  // the second field (not the output buffer)
    const double *zz;   // numerator of a for right-hand side r at zz[r * stride]
    const double *ww;   // denominator of a at ww[r * stride]
    int stride;
    int add;            // 1: out = D in + a zin (EPI 4); 0: out = zin - a D^+ in (EPI 2)
};

// A CTA stages its sites' links once and applies the operator to rb
// right-hand sides in turn (r = blockIdx.y * rb + 0 .. rb-1, below nrhs).
// EPI 0: out = D in (or D^+ in).  EPI 1: also |out_r|^2 of every right-hand
// side r: one FP64 partial per CTA (FP32 per thread) into npart;
// norm_finish_kernel adds them in a fixed order into the scalar slots.
// EPI 2: out = zu.zin - a D^+ in, and |out_r|^2 as with EPI 1.
// EPI 3: out = zu.zin - D in (a residual b - D x), no norm.
// EPI 4: out = D in + a zu.zin (CGNR's w = D p carried as D z + b w), and |out_r|^2.
// a = zz[r * stride] / ww[r * stride] (0 where the denominator is not positive).
template <bool DAG, int LS, int NT, int MINB, int EPI>
__global__ void __launch_bounds__(NT, MINB)
dslash_pair_kernel(float2 *__restrict__ out0, const float2 *__restrict__ in0, const float2 *__restrict__ U, Geom g,
                   float diag, float mf, int spb, int64_t field, double *__restrict__ npart, ZUpdate zu, int nrhs,
                   int rb) {
    constexpr bool NORM = EPI == 1 || EPI == 2 || EPI == 4;
    constexpr int TPS = LS / 2;  // threads per site
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *sL = reinterpret_cast<float4 *>(smem_raw);                 // [spb][LSTRIDE]
    int *sN = reinterpret_cast<int *>(sL + (size_t)spb * LSTRIDE);      // [spb][8]
    const int V = (int)g.V;
    const int site0 = blockIdx.x * spb;
    const int r0 = blockIdx.y * rb, r1 = min(r0 + rb, nrhs);
    // EPI >= 2: the thread's 12 components of zin are requested ahead, by
    // asynchronous copies into shared memory ([k][thread]), so that their
    // latency hides behind the hops instead of following them: those of the
    // first right-hand side before the links are staged, each next one once
    // the previous epilogue has read its own.
    float4 *sZ = reinterpret_cast<float4 *>(sN + spb * 8);
    auto request_z = [&](int r) {
        const int zs = site0 + (int)threadIdx.x / TPS;
        if ((int)threadIdx.x < spb * TPS && zs < V) {
            const float2 *zp = zu.zin + (size_t)r * (size_t)field + (size_t)zs * (12 * LS) + 2 * ((int)threadIdx.x % TPS);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const unsigned sa = (unsigned)__cvta_generic_to_shared(sZ + k * blockDim.x + threadIdx.x);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(zp + k * LS) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    if (EPI >= 2 && r0 < r1) request_z(r0);
    for (int jj = threadIdx.x; jj < spb * 8; jj += blockDim.x) {
        const int ls = jj >> 3, k = jj & 7, mu = k & 3;
        const int site = site0 + ls;
        if (site < V) {
            const int L0 = g.L[0], L1 = g.L[1], L2 = g.L[2], L3 = g.L[3];
            int cmu, Lmu, stride;
            if (mu == 0) { cmu = site % L0; Lmu = L0; stride = 1; }
            else if (mu == 1) { cmu = (site / L0) % L1; Lmu = L1; stride = L0; }
            else if (mu == 2) { cmu = (site / (L0 * L1)) % L2; Lmu = L2; stride = L0 * L1; }
            else { cmu = site / (L0 * L1 * L2); Lmu = L3; stride = L0 * L1 * L2; }
            int n = cmu + (k < 4 ? 1 : -1);
            const bool wrap = (n == Lmu) || (n < 0);
            n = (n == Lmu) ? 0 : (n < 0 ? Lmu - 1 : n);
            const int nb = site + (n - cmu) * stride;
            // two stored rows, third rebuilt as conj(row0 x row1) (det U = 1)
            const float2 *p = U + ((size_t)(k < 4 ? site : nb) * 4 + mu) * 6;
            float2 m[9];
#pragma unroll
            for (int e = 0; e < 6; ++e) m[e] = p[e];
            m[6] = conj2(cmul(m[1], m[5]) - cmul(m[2], m[4]));
            m[7] = conj2(cmul(m[2], m[3]) - cmul(m[0], m[5]));
            m[8] = conj2(cmul(m[0], m[4]) - cmul(m[1], m[3]));
            const float coef = (mu == 3 && g.ap && wrap) ? 0.5f : -0.5f;
#pragma unroll
            for (int e = 0; e < 9; ++e) {
                const float re = coef * m[e].x, im = coef * m[e].y;
                sL[ls * LSTRIDE + k * 9 + e] = make_float4(re, re, im, im);
            }
            sN[ls * 8 + k] = nb;
        }
    }
    __syncthreads();
    const int ls = threadIdx.x / TPS;
    const int j = threadIdx.x - ls * TPS;
    const int s0 = 2 * j;
    const int site = site0 + ls;
    const bool active = (ls < spb) && (site < V);
    const int row = 12 * LS;
    const int *sNs = sN + ls * 8;
    for (int rhs = r0; rhs < r1; ++rhs) {
    const float2 *__restrict__ in = in0 + (size_t)rhs * (size_t)field;
    float2 *__restrict__ out = out0 + (size_t)rhs * (size_t)field;
    // the first two hops' rows are requested together with the thread's own
    // row; each later row is requested while the hop before it computes
    float4 pa[12], pb[12], self[12];
    ldrow<LS>(pa, in + (size_t)(active ? sNs[0] : 0) * row + s0);
    ldrow<LS>(pb, in + (size_t)(active ? sNs[4] : 0) * row + s0);
    ldrow<LS>(self, in + (size_t)(active ? site : 0) * row + s0);
    // fifth dimension.  D: -P_- psi(s+1) (components 6..11), -P_+ psi(s-1)
    // (components 0..5), wrapping with +mf.  D^+: the two projectors swap.
    const int up_lo = DAG ? 0 : 6, dn_lo = DAG ? 6 : 0;
    const int lane = threadIdx.x & 31;
    const int base = lane - j;
    const int lnext = base + (j == TPS - 1 ? 0 : j + 1);
    const int lprev = base + (j == 0 ? TPS - 1 : j - 1);
    const float c_up1 = (s0 + 1 == LS - 1) ? mf : -1.f;  // s1 + 1 wraps to s = 0
    const float c_dn0 = (s0 == 0) ? mf : -1.f;           // s0 - 1 wraps to s = Ls-1
    CP acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        acc[k].re = pk(diag * self[k].x, diag * self[k].z);
        acc[k].im = pk(diag * self[k].y, diag * self[k].w);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        // from s+1: slice s0 takes own s1 (coefficient -1), slice s1 takes s0 of the next lane
        const float4 su = self[up_lo + q];
        const float nx = __shfl_sync(0xffffffffu, su.x, lnext), ny = __shfl_sync(0xffffffffu, su.y, lnext);
        acc[up_lo + q].re = add2(acc[up_lo + q].re, pk(-su.z, c_up1 * nx));
        acc[up_lo + q].im = add2(acc[up_lo + q].im, pk(-su.w, c_up1 * ny));
        // from s-1: slice s0 takes s1 of the previous lane, slice s1 takes own s0 (coefficient -1)
        const float4 sd = self[dn_lo + q];
        const float pz = __shfl_sync(0xffffffffu, sd.z, lprev), pw = __shfl_sync(0xffffffffu, sd.w, lprev);
        acc[dn_lo + q].re = add2(acc[dn_lo + q].re, pk(c_dn0 * pz, -sd.x));
        acc[dn_lo + q].im = add2(acc[dn_lo + q].im, pk(c_dn0 * pw, -sd.y));
    }
    if (!NORM && !active) continue;
    float nrm = 0.f;
    if (!NORM || active) {
        const float4 *sLs = sL + ls * LSTRIDE;
        const float fs = DAG ? 1.f : -1.f;  // sig of the forward hops
        hop2<0, false>(acc, pa, sLs + 0 * 9, fs);  ldrow<LS>(pa, in + (size_t)sNs[1] * row + s0);
        hop2<0, true>(acc, pb, sLs + 4 * 9, -fs);  ldrow<LS>(pb, in + (size_t)sNs[5] * row + s0);
        hop2<1, false>(acc, pa, sLs + 1 * 9, fs);  ldrow<LS>(pa, in + (size_t)sNs[2] * row + s0);
        hop2<1, true>(acc, pb, sLs + 5 * 9, -fs);  ldrow<LS>(pb, in + (size_t)sNs[6] * row + s0);
        hop2<2, false>(acc, pa, sLs + 2 * 9, fs);  ldrow<LS>(pa, in + (size_t)sNs[3] * row + s0);
        hop2<2, true>(acc, pb, sLs + 6 * 9, -fs);  ldrow<LS>(pb, in + (size_t)sNs[7] * row + s0);
        hop2<3, false>(acc, pa, sLs + 3 * 9, fs);
        hop2<3, true>(acc, pb, sLs + 7 * 9, -fs);
        float2 *o = out + (size_t)site * row + s0;
        float a = 1.f;
        if (EPI >= 2) {
            if (EPI == 2 || EPI == 4) {
                const double ww = zu.ww[(size_t)rhs * zu.stride];
                a = ww > 0.0 ? (float)(zu.zz[(size_t)rhs * zu.stride] / ww) : 0.f;
            }
            // each thread reads back only what its own copies wrote
            asm volatile("cp.async.wait_all;\n" ::: "memory");
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float2 re = unpk(acc[k].re), im = unpk(acc[k].im);
            if (EPI == 2 || EPI == 3) {
                const float4 z = sZ[k * blockDim.x + threadIdx.x];
                re = make_float2(fmaf(-a, re.x, z.x), fmaf(-a, re.y, z.z));
                im = make_float2(fmaf(-a, im.x, z.y), fmaf(-a, im.y, z.w));
            } else if (EPI == 4) {
                const float4 z = sZ[k * blockDim.x + threadIdx.x];
                re = make_float2(fmaf(a, z.x, re.x), fmaf(a, z.z, re.y));
                im = make_float2(fmaf(a, z.y, im.x), fmaf(a, z.w, im.y));
            }
            *reinterpret_cast<float4 *>(o + k * LS) = make_float4(re.x, im.x, re.y, im.y);
            if (NORM) nrm += re.x * re.x + im.x * im.x + re.y * re.y + im.y * im.y;
        }
    }
    // the epilogue has read this thread's staged components: request the next ones
    if (EPI >= 2 && rhs + 1 < r1) request_z(rhs + 1);
    if (NORM) {
        __shared__ double wsum[4];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
        const int warp = threadIdx.x >> 5;
        if (lane == 0) wsum[warp] = (double)nrm;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int w = 0; w < ((int)blockDim.x + 31) >> 5; ++w) t += wsum[w];
            npart[(size_t)rhs * gridDim.x + blockIdx.x] = t;
        }
        __syncthreads();  // wsum is rewritten for the next right-hand side
    }
    }
}

// nslot[r * nstride] = sum of the nb CTA partials of right-hand side r = blockIdx.x (fixed order)
__global__ void __launch_bounds__(1024) norm_finish_kernel(const double *__restrict__ npart, double *__restrict__ nslot,
                                                           int nstride, int nb) {
    __shared__ double red[32];
    const double *pr = npart + (size_t)blockIdx.x * nb;
    double t = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) t += pr[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += red[w];
        nslot[(size_t)blockIdx.x * nstride] = u;
    }
}

// CTAs of 64 threads, 8 per SM (minb = 8, the default: measured 2-3% faster
// than 128 threads x 4, by locality of the smaller site tiles) or of 128
// threads, 4 per SM (minb = 4); 128 registers either way.
template <int LS>
void launch_ls(dwf_ctx *c, float2 *out, const float2 *in, bool dag, int nrhs, int minb, double *nslot, int nstride,
               const ZUpdate *zu) {
    const Geom &g = c->g;
    constexpr int TPS = LS / 2;
    int spb = (minb == 4 ? 128 : 64) / TPS;
    const size_t per_site = LSTRIDE * sizeof(float4) + 8 * sizeof(int);
    // shared memory per site: staged links and neighbour table, and with zu
    // the TPS threads' staged components of zin (12 float4 each)
    const size_t per_site_all = per_site + (zu ? (size_t)TPS * 12 * sizeof(float4) : 0);
    const int max_spb = (int)((46 * 1024) / per_site_all);
    if (spb > max_spb) spb = max_spb;
    // whole warps: the s-neighbour shuffles and the norm reduction use full masks
    if (TPS < 32) spb = std::max(32 / TPS, spb / (32 / TPS) * (32 / TPS));
    const int threads = spb * TPS;
    // right-hand sides per CTA: the links staged once serve up to 4 of them
    // (measured 3-4 % faster for the plain and norm kernels; the kernels that
    // stage a second field run one right-hand side per CTA, 5 % faster so)
    const int rb = zu ? 1 : std::min(nrhs, 4);
    dim3 grid((unsigned)((g.V + spb - 1) / spb), (unsigned)((nrhs + rb - 1) / rb));
    size_t smem = (size_t)spb * per_site;
    if (zu) smem += (size_t)threads * 12 * sizeof(float4);  // the staged zin components
    DWF_REQUIRE(smem <= 48 * 1024, DWF_EINVAL, "paired Dslash: shared memory above the default 48 KB");
    int64_t field = g.V * g.Ls * 12;
    float diag = (float)(5.0 - c->M5), mf = (float)c->mf;
    const float2 *U = c->U32.as<float2>();
    double *npart = nullptr;
    if (nslot) {
        const size_t pb = sizeof(double) * (size_t)grid.x * nrhs;
        if (c->dn_part.bytes < pb) c->dn_part.alloc(pb);
        npart = c->dn_part.as<double>();
    }
    const ZUpdate z = zu ? *zu : ZUpdate{nullptr, nullptr, nullptr, 0, 0};
#define PL(D, NT, M, E) dslash_pair_kernel<D, LS, NT, M, E><<<grid, threads, smem, c->stream>>>(out, in, U, g, diag, mf, \
                                                                                                 spb, field, npart, z, \
                                                                                                 nrhs, rb)
    if (zu && !nslot) {
        if (minb == 4) PL(false, 128, 4, 3); else PL(false, 64, 8, 3);
    } else if (zu && zu->add) {
        if (minb == 4) PL(false, 128, 4, 4); else PL(false, 64, 8, 4);
        DWF_CHECK_LAUNCH();
        norm_finish_kernel<<<nrhs, 1024, 0, c->stream>>>(npart, nslot, nstride, (int)grid.x);
    } else if (zu) {
        if (minb == 4) PL(true, 128, 4, 2); else PL(true, 64, 8, 2);
        DWF_CHECK_LAUNCH();
        norm_finish_kernel<<<nrhs, 1024, 0, c->stream>>>(npart, nslot, nstride, (int)grid.x);
    } else if (nslot) {
        if (dag) { if (minb == 4) PL(true, 128, 4, 1); else PL(true, 64, 8, 1); }
        else { if (minb == 4) PL(false, 128, 4, 1); else PL(false, 64, 8, 1); }
        DWF_CHECK_LAUNCH();
        norm_finish_kernel<<<nrhs, 1024, 0, c->stream>>>(npart, nslot, nstride, (int)grid.x);
    } else {
        if (dag) { if (minb == 4) PL(true, 128, 4, 0); else PL(true, 64, 8, 0); }
        else { if (minb == 4) PL(false, 128, 4, 0); else PL(false, 64, 8, 0); }
    }
#undef PL
    DWF_CHECK_LAUNCH();
}

}  // namespace

// true when the paired FP32 kernel handles this fifth extent
bool dslash_pair_supported(int Ls) { return Ls == 4 || Ls == 8 || Ls == 16 || Ls == 32 || Ls == 64; }

void dslash_pair_f32(dwf_ctx *c, float2 *out, const float2 *in, bool dag, int nrhs, int minb, double *nslot,
                     int nstride, const float2 *zin, const double *zz, const double *ww, bool add) {
    const ZUpdate zu{zin, zz, ww, nstride, add ? 1 : 0};
    const ZUpdate *zp = zin ? &zu : nullptr;
    switch (c->g.Ls) {
        case 4: launch_ls<4>(c, out, in, dag, nrhs, minb, nslot, nstride, zp); break;
        case 8: launch_ls<8>(c, out, in, dag, nrhs, minb, nslot, nstride, zp); break;
        case 16: launch_ls<16>(c, out, in, dag, nrhs, minb, nslot, nstride, zp); break;
        case 32: launch_ls<32>(c, out, in, dag, nrhs, minb, nslot, nstride, zp); break;
        case 64: launch_ls<64>(c, out, in, dag, nrhs, minb, nslot, nstride, zp); break;
        default: throw Error{DWF_EINVAL, "paired Dslash needs Ls in {4, 8, 16, 32, 64}"};
    }
}

}  // namespace dwf
