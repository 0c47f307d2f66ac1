// Spin-projected hopping terms of the Wilson part of the domain-wall
// operator, shared by the Dslash and the coarse-operator construction.
//
// The hop along mu multiplies by (1 + sig*g_mu) (sig = -1 forward / +1
// backward for D; reversed for D^+).  That matrix has rank 2: two "half
// spinor" rows h0, h1 are formed, multiplied by the link, and rows 2, 3 of
// the result are fixed multiples of h0, h1 in the chiral basis with
// g_5 = diag(1,1,-1,-1):
//   g_x: h0 = p0 + sig i p3, h1 = p1 + sig i p2;  row2 = -sig i h1, row3 = -sig i h0
//   g_y: h0 = p0 - sig p3,   h1 = p1 + sig p2;    row2 =  sig h1,   row3 = -sig h0
//   g_z: h0 = p0 + sig i p2, h1 = p1 - sig i p3;  row2 = -sig i h0, row3 =  sig i h1
//   g_t: h0 = p0 + sig p2,   h1 = p1 + sig p3;    row2 =  sig h0,   row3 =  sig h1
#pragma once
#include "dwf_internal.cuh"

namespace dwf {

template <typename R> struct LinkIO;

template <> struct LinkIO<double> {
    // full 3x3, [site][mu][9]
    static __device__ __forceinline__ void load(const double2 *U, int64_t site, int mu, double2 m[9]) {
        const double2 *p = U + (site * 4 + mu) * 9;
#pragma unroll
        for (int e = 0; e < 9; ++e) m[e] = p[e];
    }
};

template <> struct LinkIO<float> {
    // two rows, [site][mu][6]; third row rebuilt (det U = 1)
    static __device__ __forceinline__ void load(const float2 *U, int64_t site, int mu, float2 m[9]) {
        const float2 *p = U + (site * 4 + mu) * 6;
#pragma unroll
        for (int e = 0; e < 6; ++e) m[e] = p[e];
        m[6] = conj2(cmul(m[1], m[5]) - cmul(m[2], m[4]));
        m[7] = conj2(cmul(m[2], m[3]) - cmul(m[0], m[5]));
        m[8] = conj2(cmul(m[0], m[4]) - cmul(m[1], m[3]));
    }
};

template <int MU, typename T> __device__ __forceinline__ void project(const T p[12], int sig, T h[6]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T p0 = p[a], p1 = p[3 + a], p2 = p[6 + a], p3 = p[9 + a];
        T s0, s1;
        if (MU == 0) { s0 = mul_i(p3); s1 = mul_i(p2); }
        if (MU == 1) { s0 = mk<decltype(p0.x)>(-p3.x, -p3.y); s1 = p2; }
        if (MU == 2) { s0 = mul_i(p2); s1 = mk<decltype(p0.x)>(p3.y, -p3.x); }  // -i p3
        if (MU == 3) { s0 = p2; s1 = p3; }
        if (sig > 0) { h[a] = p0 + s0; h[3 + a] = p1 + s1; }
        else         { h[a] = p0 - s0; h[3 + a] = p1 - s1; }
    }
}

template <int MU, typename T, typename R>
__device__ __forceinline__ void reconstruct_add(T acc[12], const T u[6], int sig, R coef) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T u0 = coef * u[a], u1 = coef * u[3 + a];
        acc[a] = acc[a] + u0;
        acc[3 + a] = acc[3 + a] + u1;
        T r2, r3;
        if (MU == 0) { r2 = mk<R>(u1.y, -u1.x); r3 = mk<R>(u0.y, -u0.x); }   // -i u1, -i u0
        if (MU == 1) { r2 = u1; r3 = mk<R>(-u0.x, -u0.y); }
        if (MU == 2) { r2 = mk<R>(u0.y, -u0.x); r3 = mul_i(u1); }            // -i u0, i u1
        if (MU == 3) { r2 = u0; r3 = u1; }
        if (sig > 0) { acc[6 + a] = acc[6 + a] + r2; acc[9 + a] = acc[9 + a] + r3; }
        else         { acc[6 + a] = acc[6 + a] - r2; acc[9 + a] = acc[9 + a] - r3; }
    }
}

// one 4D hop: acc += coef * (1 + sig g_mu) M h   with M = U or U^+
template <int MU, bool ADJ, typename R>
__device__ __forceinline__ void hop(C<R> acc[12], const C<R> *__restrict__ in, int64_t y, int Ls, int s,
                                    const C<R> *m, int sig, R coef) {
    C<R> p[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = in[(y * 12 + k) * Ls + s];
    C<R> h[6], u[6];
    project<MU>(p, sig, h);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C<R> z = mk<R>(0, 0);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (ADJ) cfmac(z, m[b * 3 + a], h[sp * 3 + b]);
                else cfma(z, m[a * 3 + b], h[sp * 3 + b]);
            }
            u[sp * 3 + a] = z;
        }
    reconstruct_add<MU>(acc, u, sig, coef);
}


}  // namespace dwf
