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
#include "spin.cuh"

namespace dwf {

namespace {

template <int MU, bool DAG, typename R>
__device__ __forceinline__ void hops_mu(C<R> acc[12], const C<R> *__restrict__ in, const Geom &g,
                                        const int c[4], int64_t site, int s, const C<R> *sUsite) {
    // forward neighbour x + mu
    {
        int cc[4] = {c[0], c[1], c[2], c[3]};
        cc[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
        R coef = (MU == 3 && g.ap && c[3] == g.L[3] - 1) ? R(0.5) : R(-0.5);
        hop<MU, false, R>(acc, in, site_index(g, cc), g.Ls, s, sUsite + MU * 9, DAG ? +1 : -1, coef);
    }
    // backward neighbour x - mu
    {
        int cc[4] = {c[0], c[1], c[2], c[3]};
        cc[MU] = (c[MU] == 0) ? g.L[MU] - 1 : c[MU] - 1;
        R coef = (MU == 3 && g.ap && c[3] == 0) ? R(0.5) : R(-0.5);
        hop<MU, true, R>(acc, in, site_index(g, cc), g.Ls, s, sUsite + (4 + MU) * 9, DAG ? -1 : +1, coef);
    }
}

template <typename R, bool DAG>
__global__ void __launch_bounds__(256) dslash_kernel(C<R> *__restrict__ out, const C<R> *__restrict__ in,
                                                     const C<R> *__restrict__ U, Geom g, R diag, R mf,
                                                     int spb, int64_t field) {
    extern __shared__ unsigned char smem_raw[];
    C<R> *sU = reinterpret_cast<C<R> *>(smem_raw);
    const int64_t site0 = (int64_t)blockIdx.x * spb;
    const int64_t rhs_off = (int64_t)blockIdx.y * field;
    in += rhs_off;
    out += rhs_off;
    // stage the 8 links of every site of this CTA
    for (int j = threadIdx.x; j < spb * 8; j += blockDim.x) {
        int ls = j >> 3, k = j & 7, mu = k & 3;
        int64_t site = site0 + ls;
        if (site < g.V) {
            int64_t lsite = site;
            if (k >= 4) {
                int c[4];
                site_coords(g, site, c);
                c[mu] = (c[mu] == 0) ? g.L[mu] - 1 : c[mu] - 1;
                lsite = site_index(g, c);
            }
            C<R> m[9];
            LinkIO<R>::load(U, lsite, mu, m);
#pragma unroll
            for (int e = 0; e < 9; ++e) sU[(ls * 8 + k) * 9 + e] = m[e];
        }
    }
    __syncthreads();
    const int ls = threadIdx.x / g.Ls;
    const int s = threadIdx.x - ls * g.Ls;
    const int64_t site = site0 + ls;
    if (ls >= spb || site >= g.V) return;
    int c[4];
    site_coords(g, site, c);
    const C<R> *sUsite = sU + ls * 8 * 9;
    C<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = diag * in[(site * 12 + k) * g.Ls + s];
    hops_mu<0, DAG, R>(acc, in, g, c, site, s, sUsite);
    hops_mu<1, DAG, R>(acc, in, g, c, site, s, sUsite);
    hops_mu<2, DAG, R>(acc, in, g, c, site, s, sUsite);
    hops_mu<3, DAG, R>(acc, in, g, c, site, s, sUsite);
    // fifth dimension: D has -P_- psi(s+1) and -P_+ psi(s-1) (wrap: +mf);
    // D^+ has -P_+ psi(s+1) and -P_- psi(s-1) (wrap: +mf).
    {
        int sp = (s == g.Ls - 1) ? 0 : s + 1;
        R cp = (s == g.Ls - 1) ? mf : R(-1);
        int sm = (s == 0) ? g.Ls - 1 : s - 1;
        R cm = (s == 0) ? mf : R(-1);
        const int up_lo = DAG ? 0 : 6;   // components taken from s+1
        const int dn_lo = DAG ? 6 : 0;   // components taken from s-1
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            acc[up_lo + k] = acc[up_lo + k] + cp * in[(site * 12 + up_lo + k) * g.Ls + sp];
            acc[dn_lo + k] = acc[dn_lo + k] + cm * in[(site * 12 + dn_lo + k) * g.Ls + sm];
        }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) out[(site * 12 + k) * g.Ls + s] = acc[k];
}

template <typename R>
void launch(dwf_ctx *c, C<R> *out, const C<R> *in, const C<R> *U, bool dag, int nrhs) {
    const Geom &g = c->g;
    int spb = g.Ls >= 128 ? 1 : 128 / g.Ls;
    int threads = spb * g.Ls;
    dim3 grid((unsigned)((g.V + spb - 1) / spb), (unsigned)nrhs);
    size_t smem = (size_t)spb * 8 * 9 * sizeof(C<R>);
    int64_t field = g.V * g.Ls * 12;
    if (dag)
        dslash_kernel<R, true><<<grid, threads, smem, c->stream>>>(out, in, U, g, R(5.0 - c->M5), R(c->mf), spb, field);
    else
        dslash_kernel<R, false><<<grid, threads, smem, c->stream>>>(out, in, U, g, R(5.0 - c->M5), R(c->mf), spb, field);
    DWF_CHECK_LAUNCH();
}

}  // namespace

void dslash(dwf_ctx *c, double2 *out, const double2 *in, bool dag, int nrhs) {
    launch<double>(c, out, in, c->U64.as<double2>(), dag, nrhs);
    c->applies64 += nrhs;
}

void dslash(dwf_ctx *c, float2 *out, const float2 *in, bool dag, int nrhs) {
    launch<float>(c, out, in, c->U32.as<float2>(), dag, nrhs);
    c->applies32 += nrhs;
}

}  // namespace dwf
