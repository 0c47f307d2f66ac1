// Fine Shamir domain-wall operator D and D^+ (Sec. 2 of Cohen-Brower-Clark-
// Osborn: the domain-wall operator with fifth dimension Ls; Sec. 4: every
// output site reads itself and its 10 unit-distance neighbours in 5D).
//
// Layout: fermion fields are [site][spin*3+colour][s] complex (s fastest),
// so the Ls threads of one 4D site read consecutive addresses of every
// component (coalesced).  Each CTA covers `spb` whole 4D sites x Ls.  The 8
// links a 4D site needs (U_mu(x) and U_mu(x-mu)) are loaded once per CTA into
// shared memory and reused by all Ls threads of the site; the FP32 copy
// stores two rows per link and rebuilds the third as conj(row0 x row1).
//
// Spin projection: see spin.cuh.
#include <cstdlib>

#include "spin.cuh"

namespace dwf {

namespace {

// One 4D hop for the thread's (site, s): spinor row `p` (already offset to s),
// component stride LS; the staged link `m` already carries the hop
// coefficient (-1/2, or +1/2 across an antiperiodic t boundary).
template <int MU, bool ADJ, typename R, int LS>
__device__ __forceinline__ void hop_row(C<R> acc[12], const C<R> *__restrict__ p, int ls_rt, const C<R> *m, int sig) {
    const int Ls = LS > 0 ? LS : ls_rt;
    C<R> v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = p[k * Ls];
    C<R> h[6], u[6];
    project<MU>(v, sig, h);
    C<R> mm[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) mm[e] = m[e];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C<R> z = mk<R>(0, 0);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (ADJ) cfmac(z, mm[b * 3 + a], h[sp * 3 + b]);
                else cfma(z, mm[a * 3 + b], h[sp * 3 + b]);
            }
            u[sp * 3 + a] = z;
        }
    reconstruct_add<MU>(acc, u, sig, R(1));
}

// CTA = spb whole 4D sites x Ls threads.  Phase 1 (spb*8 threads): each
// stages one link (U_mu(x) forward, U_mu(x-mu) backward), scaled by its hop
// coefficient, into shared memory with the neighbour's site index.  Phase 2:
// every thread computes its 5D site.  SHFL: the Ls threads of a site sit
// inside one warp (Ls divides 32) and the fifth-dimension neighbours come
// from shuffles.  LS > 0: the fifth extent is a compile-time constant, so
// every component load uses an immediate offset.
template <typename R, bool DAG, bool SHFL, int LS, int MINB>
__global__ void __launch_bounds__(128, MINB)
dslash_kernel(C<R> *__restrict__ out, const C<R> *__restrict__ in, const C<R> *__restrict__ U, Geom g, R diag, R mf,
              int spb, int64_t field) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<R> *sU = reinterpret_cast<C<R> *>(smem_raw);               // [spb][8][10] (9 used)
    int *sN = reinterpret_cast<int *>(sU + (size_t)spb * 80);       // [spb][8]
    const int Ls = LS > 0 ? LS : g.Ls;
    const int V = (int)g.V;
    const int site0 = blockIdx.x * spb;
    const size_t rhs_off = (size_t)blockIdx.y * (size_t)field;
    in += rhs_off;
    out += rhs_off;
    for (int j = threadIdx.x; j < spb * 8; j += blockDim.x) {
        const int ls = j >> 3, k = j & 7, mu = k & 3;
        const int site = site0 + ls;
        if (site < V) {
            // coordinate along mu, extent and site stride of direction mu
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
            C<R> m[9];
            LinkIO<R>::load(U, k < 4 ? site : nb, mu, m);
            const R coef = (mu == 3 && g.ap && wrap) ? R(0.5) : R(-0.5);
#pragma unroll
            for (int e = 0; e < 9; ++e) sU[(ls * 8 + k) * 10 + e] = coef * m[e];
            sN[ls * 8 + k] = nb;
        }
    }
    __syncthreads();
    const int ls = threadIdx.x / Ls;
    const int s = threadIdx.x - ls * Ls;
    const int site = site0 + ls;
    const bool active = (ls < spb) && (site < V);
    if (!SHFL && !active) return;
    const int row = 12 * Ls;
    C<R> acc[12], self[12];
    if (active) {
        const C<R> *p = in + (size_t)site * row + s;
#pragma unroll
        for (int k = 0; k < 12; ++k) self[k] = p[k * Ls];
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) self[k] = mk<R>(0, 0);
    }
    // fifth dimension: D has -P_- psi(s+1) and -P_+ psi(s-1) (wrap: +mf);
    // D^+ has -P_+ psi(s+1) and -P_- psi(s-1) (wrap: +mf).
    const int up_lo = DAG ? 0 : 6;   // components taken from s+1
    const int dn_lo = DAG ? 6 : 0;   // components taken from s-1
    const R cp = (s == Ls - 1) ? mf : R(-1);
    const R cm = (s == 0) ? mf : R(-1);
    C<R> up[6], dn[6];
    if (SHFL) {
        const int lane = threadIdx.x & 31;
        const int base = lane - s;
        const int lup = base + ((s == Ls - 1) ? 0 : s + 1);
        const int ldn = base + ((s == 0) ? Ls - 1 : s - 1);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            up[k].x = __shfl_sync(0xffffffffu, self[up_lo + k].x, lup);
            up[k].y = __shfl_sync(0xffffffffu, self[up_lo + k].y, lup);
            dn[k].x = __shfl_sync(0xffffffffu, self[dn_lo + k].x, ldn);
            dn[k].y = __shfl_sync(0xffffffffu, self[dn_lo + k].y, ldn);
        }
        if (!active) return;
    } else {
        const C<R> *p = in + (size_t)site * row;
        const int sp = (s == Ls - 1) ? 0 : s + 1;
        const int sm = (s == 0) ? Ls - 1 : s - 1;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            up[k] = p[(up_lo + k) * Ls + sp];
            dn[k] = p[(dn_lo + k) * Ls + sm];
        }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = diag * self[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        acc[up_lo + k] = acc[up_lo + k] + cp * up[k];
        acc[dn_lo + k] = acc[dn_lo + k] + cm * dn[k];
    }
    const C<R> *sUs = sU + ls * 80;
    const int *sNs = sN + ls * 8;
    const int fs = DAG ? +1 : -1;  // sig of the forward hops
    hop_row<0, false, R, LS>(acc, in + (size_t)sNs[0] * row + s, Ls, sUs + 0 * 10, fs);
    hop_row<0, true, R, LS>(acc, in + (size_t)sNs[4] * row + s, Ls, sUs + 4 * 10, -fs);
    hop_row<1, false, R, LS>(acc, in + (size_t)sNs[1] * row + s, Ls, sUs + 1 * 10, fs);
    hop_row<1, true, R, LS>(acc, in + (size_t)sNs[5] * row + s, Ls, sUs + 5 * 10, -fs);
    hop_row<2, false, R, LS>(acc, in + (size_t)sNs[2] * row + s, Ls, sUs + 2 * 10, fs);
    hop_row<2, true, R, LS>(acc, in + (size_t)sNs[6] * row + s, Ls, sUs + 6 * 10, -fs);
    hop_row<3, false, R, LS>(acc, in + (size_t)sNs[3] * row + s, Ls, sUs + 3 * 10, fs);
    hop_row<3, true, R, LS>(acc, in + (size_t)sNs[7] * row + s, Ls, sUs + 7 * 10, -fs);
    C<R> *o = out + (size_t)site * row + s;
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k * Ls] = acc[k];
}

template <typename R>
void launch(dwf_ctx *c, C<R> *out, const C<R> *in, const C<R> *U, bool dag, int nrhs) {
    const Geom &g = c->g;
    DWF_REQUIRE(g.V * g.Ls * 12 < (int64_t)1 << 31 && g.V < (int64_t)1 << 31, DWF_EINVAL,
                "lattice too large for 32-bit element offsets of one field");
    // sites per CTA: about 128 threads, staging within 46 KB of shared memory
    int spb = g.Ls >= 128 ? 1 : 128 / g.Ls;
    const size_t per_site = 80 * sizeof(C<R>) + 8 * sizeof(int);
    const int max_spb = (int)((46 * 1024) / per_site);
    if (spb > max_spb) spb = max_spb;
    const bool shfl = (32 % g.Ls) == 0;
    int threads = spb * g.Ls;
    if (shfl) threads = (threads + 31) / 32 * 32;  // whole warps for the shuffles
    dim3 grid((unsigned)((g.V + spb - 1) / spb), (unsigned)nrhs);
    size_t smem = (size_t)spb * per_site;
    int64_t field = g.V * g.Ls * 12;
    R diag = R(5.0 - c->M5), mf = R(c->mf);
    // register budget: 8 CTAs/SM (64 registers, small spills) or 6 (80);
    // DWF_DSLASH_MINB=6 selects the latter
    static const int minb = [] {
        const char *e = getenv("DWF_DSLASH_MINB");
        return (e && atoi(e) == 6) ? 6 : 8;
    }();
#define DLM(D, S, L, M) dslash_kernel<R, D, S, L, M><<<grid, threads, smem, c->stream>>>(out, in, U, g, diag, mf, spb, field)
#define DL(D, S, L)                                          \
    do {                                                     \
        if constexpr (sizeof(R) == 8) DLM(D, S, L, 4);       \
        else if (minb == 6) DLM(D, S, L, 6);                 \
        else DLM(D, S, L, 8);                                \
    } while (0)
    if (g.Ls == 16) {
        if (dag) DL(true, true, 16); else DL(false, true, 16);
    } else if (g.Ls == 8) {
        if (dag) DL(true, true, 8); else DL(false, true, 8);
    } else if (dag) {
        if (shfl) DL(true, true, 0); else DL(true, false, 0);
    } else {
        if (shfl) DL(false, true, 0); else DL(false, false, 0);
    }
#undef DLM
#undef DL
    DWF_CHECK_LAUNCH();
}

}  // namespace

void dslash(dwf_ctx *c, double2 *out, const double2 *in, bool dag, int nrhs) {
    ProfScope ps(c, K_DSLASH_F64, nrhs);
    launch<double>(c, out, in, c->U64.as<double2>(), dag, nrhs);
    c->applies64 += nrhs;
}

bool dslash_pair_supported(int Ls);
// zin with nslot: out = zin - a D^+ in (add: out = D in + a zin), a = zz[r * nstride] / ww[r * nstride]
// per right-hand side r; zin without nslot: out = zin - D in
void dslash_pair_f32(dwf_ctx *c, float2 *out, const float2 *in, bool dag, int nrhs, int minb, double *nslot,
                     int nstride, const float2 *zin = nullptr, const double *zz = nullptr, const double *ww = nullptr,
                     bool add = false);

namespace {
// two slices per thread with packed FP32x2 arithmetic where Ls allows;
// DWF_DSLASH_PAIR=0 selects the one-slice kernel, DWF_DSLASH_PAIR_MINB=4 the
// 128-thread CTAs instead of the default 64-thread ones (8 per SM)
int pair_minb() {
    static const int v = [] {
        const char *e = getenv("DWF_DSLASH_PAIR");
        if (e && atoi(e) == 0) return 0;
        const char *m = getenv("DWF_DSLASH_PAIR_MINB");
        return (m && atoi(m) == 4) ? 4 : 8;
    }();
    return v;
}
}  // namespace

void dslash(dwf_ctx *c, float2 *out, const float2 *in, bool dag, int nrhs) {
    ProfScope ps(c, K_DSLASH_F32, nrhs);
    if (pair_minb() && dslash_pair_supported(c->g.Ls)) {
        dslash_pair_f32(c, out, in, dag, nrhs, pair_minb(), nullptr, 0);
        c->applies32 += nrhs;
        return;
    }
    launch<float>(c, out, in, c->U32.as<float2>(), dag, nrhs);
    c->applies32 += nrhs;
}

bool dslash_norm_fused(dwf_ctx *c) { return pair_minb() && dslash_pair_supported(c->g.Ls); }

void dslash_norm(dwf_ctx *c, float2 *out, const float2 *in, bool dag, int nrhs, int slot, int stride) {
    DWF_REQUIRE(dslash_norm_fused(c), DWF_EINVAL, "fused Dslash norm needs the paired kernel");
    ProfScope ps(c, K_DSLASH_F32, nrhs);
    dslash_pair_f32(c, out, in, dag, nrhs, pair_minb(), c->scal.as<double>() + slot, stride);
    c->applies32 += nrhs;
}

void dslash_residual(dwf_ctx *c, float2 *res, const float2 *x, const float2 *b, int nrhs) {
    DWF_REQUIRE(dslash_norm_fused(c), DWF_EINVAL, "fused residual needs the paired kernel");
    DWF_REQUIRE(res != x && res != b, DWF_EINVAL, "residual: output must not alias an input");
    ProfScope ps(c, K_DSLASH_F32_Z, nrhs);
    dslash_pair_f32(c, res, x, false, nrhs, pair_minb(), nullptr, 0, b);
    c->applies32 += nrhs;
}

void dslash_wupdate(dwf_ctx *c, float2 *wout, const float2 *z, const float2 *win, int nrhs, int slot, int stride,
                    int inum, int iden) {
    DWF_REQUIRE(dslash_norm_fused(c), DWF_EINVAL, "fused direction update needs the paired kernel");
    DWF_REQUIRE(wout != win && wout != z, DWF_EINVAL, "direction update: output must not alias an input");
    ProfScope ps(c, K_DSLASH_F32_Z, nrhs);
    double *s = c->scal.as<double>();
    dslash_pair_f32(c, wout, z, false, nrhs, pair_minb(), s + slot, stride, win, s + inum, s + iden, true);
    c->applies32 += nrhs;
}

void dslash_zupdate(dwf_ctx *c, float2 *zout, const float2 *w, const float2 *zin, int nrhs, int slot, int stride,
                    int izz, int iww) {
    DWF_REQUIRE(dslash_norm_fused(c), DWF_EINVAL, "fused residual update needs the paired kernel");
    DWF_REQUIRE(zout != zin && zout != w, DWF_EINVAL, "residual update: output must not alias an input");
    ProfScope ps(c, K_DSLASH_F32_Z, nrhs);
    double *s = c->scal.as<double>();
    dslash_pair_f32(c, zout, w, true, nrhs, pair_minb(), s + slot, stride, zin, s + izz, s + iww);
    c->applies32 += nrhs;
}

}  // namespace dwf
