// Learned near-null proposal: a gauge-covariant convolutional network, its
// backward pass, the block-projection loss against the adaptive setup's
// vectors and an Adam step (the definitions are in include/dwfnet.h; the
// paper has no counterpart, its setup relaxes on D x = 0, Sec. 2).
//
// Activations are planar complex FP32 matrices [rows][V*3] (row = channel*4
// + spin, column = site*3 + colour), so every layer is
//   transports (a stencil kernel) -> one complex GEMM -> the gate,
// and every backward step is the adjoint GEMM, the adjoint transports and
// the gate's derivative.  The GEMM is a plain shared-memory tiled SIMT
// kernel with split-K partial sums (the network is small and off the solve's
// hot path; it runs once per setup).
#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "dwf_internal.cuh"
#include "dwfnet.h"
#include "mg.cuh"

struct dwf_net {
    dwf_net_shape sh;
    int device = 0;
    int64_t nparams = 0;
    std::vector<int64_t> off;  // parameter group offsets (layers..., head)
    dwf::DevBuf P, G, M1, M2;  // parameters, gradient, Adam moments (FP32 complex)
    // inference weights: BF16-rounded copy of P when the weight precision is BF16
    dwf::DevBuf Pi;
    dwf_prec wprec = DWF_F32;
    bool pi_valid = false;
    int adam_t = 0;
    bool have_grad = false;
    // workspaces for one lattice volume and batch (B fields side by side in
    // the columns: column (b*V + site)*3 + colour)
    int64_t V = -1;
    int B = 0;
    float oscale = 1.f;  // head output scale: 1, or 1/alpha in refinement mode
    std::vector<dwf::DevBuf> h, a, S;
    dwf::DevBuf vh, v, F, R, gvh, gh, ga, yt, gws, gpart, gram, Y, info, lpart, lval, in64;
};

namespace dwf {

namespace {

constexpr uint32_t STREAM_NETWORK = 7;
constexpr int NT = 256;

unsigned grid1(dwf_ctx *c, int64_t n) {
    int64_t b = (n + NT - 1) / NT;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)c->sm_count * 16));
}

// ---------------------------------------------------------------------------
// complex GEMM  C[M][N] = op(A) op(B)
//   opA = 0: op(A)[m][k] = A[m*lda + k];   opA = 1: conj(A[k*lda + m])
//   opB = 0: op(B)[k][n] = B[k*ldb + n];   opB = 1: conj(B[n*ldb + k])
// blockIdx.z takes the K range [z*kchunk, (z+1)*kchunk) and writes its own
// partial product at C + z*cstride.
// ---------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 8;

__global__ void __launch_bounds__(256) cgemm_kernel(float2 *__restrict__ C, const float2 *__restrict__ A,
                                                    const float2 *__restrict__ B, int M, int N, int K, int64_t lda,
                                                    int64_t ldb, int opA, int opB, int kchunk, int64_t cstride) {
    __shared__ float2 As[GBK][GBM];
    __shared__ float2 Bs[GBK][GBN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = kbeg; k0 < kend; k0 += GBK) {
        for (int e = tid; e < GBK * GBM; e += 256) {
            int kk, mm;
            if (opA == 0) { mm = e / GBK; kk = e - mm * GBK; }
            else { kk = e / GBM; mm = e - kk * GBM; }
            const int m = m0 + mm, k = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (m < M && k < kend) v = opA == 0 ? A[(int64_t)m * lda + k] : conj2(A[(int64_t)k * lda + m]);
            As[kk][mm] = v;
        }
        for (int e = tid; e < GBK * GBN; e += 256) {
            int kk, nn;
            if (opB == 0) { kk = e / GBN; nn = e - kk * GBN; }
            else { nn = e / GBK; kk = e - nn * GBK; }
            const int n = n0 + nn, k = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (n < N && k < kend) v = opB == 0 ? B[(int64_t)k * ldb + n] : conj2(B[(int64_t)n * ldb + k]);
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            float2 av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], av[i], bv[j]);
        }
        __syncthreads();
    }
    float2 *Cz = C + (int64_t)blockIdx.z * cstride;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
            if (m < M && n < N) Cz[(int64_t)m * N + n] = acc[i][j];
        }
}

// C = sum of nz partial products (FP64 sums, fixed order)
__global__ void sum_partials_kernel(float2 *__restrict__ C, const float2 *__restrict__ P, int nz, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x = 0, y = 0;
        for (int z = 0; z < nz; ++z) {
            float2 v = P[(int64_t)z * n + i];
            x += v.x;
            y += v.y;
        }
        C[i] = make_float2((float)x, (float)y);
    }
}

// ---------------------------------------------------------------------------
// parallel transports: S[d][i][x][c] = (T_d h)[i][x][c], d = 0..8
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t shifted(const Geom &g, const int co[4], int mu, int dir) {
    int c[4] = {co[0], co[1], co[2], co[3]};
    c[mu] += dir;
    if (c[mu] == g.L[mu]) c[mu] = 0;
    if (c[mu] < 0) c[mu] = g.L[mu] - 1;
    return site_index(g, c);
}

__global__ void transport_kernel(float2 *__restrict__ S, const float2 *__restrict__ h, const double2 *__restrict__ U,
                                 Geom g, int nrow, int B) {
    const int64_t V = g.V, cols = (int64_t)B * V * 3, plane = (int64_t)nrow * cols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)nrow * B * V;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / (B * V), xb = t - i * B * V;
        const int64_t b = xb / V, x = xb - b * V;
        int co[4];
        site_coords(g, x, co);
        const float2 *hi = h + i * cols + b * V * 3;
        float2 *So = S + i * cols + xb * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) So[c] = hi[x * 3 + c];
        for (int mu = 0; mu < 4; ++mu) {
            const int64_t xp = shifted(g, co, mu, +1), xm = shifted(g, co, mu, -1);
            const double2 *u = U + (x * 4 + mu) * 9;   // U_mu(x)
            const double2 *um = U + (xm * 4 + mu) * 9; // U_mu(x - mu)
            float2 hp[3], hm[3];
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) { hp[bb] = hi[xp * 3 + bb]; hm[bb] = hi[xm * 3 + bb]; }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float2 sp = make_float2(0.f, 0.f), sm = make_float2(0.f, 0.f);
#pragma unroll
                for (int bb = 0; bb < 3; ++bb) {
                    cfma(sp, cvt<float2, double2>(u[a * 3 + bb]), hp[bb]);    // U(x)[a][b] h(x+mu)[b]
                    cfmac(sm, cvt<float2, double2>(um[bb * 3 + a]), hm[bb]);  // conj(U(x-mu)[b][a]) h(x-mu)[b]
                }
                So[(1 + 2 * mu) * plane + a] = sp;
                So[(2 + 2 * mu) * plane + a] = sm;
            }
        }
    }
}

// gh[i][x] = sum_d (T_d^+ Y_d)(x):  T_{+mu}^+ y(x) = U_mu(x-mu)^+ y(x-mu),
// T_{-mu}^+ y(x) = U_mu(x) y(x+mu)
__global__ void transport_adj_kernel(float2 *__restrict__ gh, const float2 *__restrict__ Y,
                                     const double2 *__restrict__ U, Geom g, int nrow, int B) {
    const int64_t V = g.V, cols = (int64_t)B * V * 3, plane = (int64_t)nrow * cols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)nrow * B * V;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / (B * V), xb = t - i * B * V;
        const int64_t b = xb / V, x = xb - b * V;
        int co[4];
        site_coords(g, x, co);
        const float2 *Yi = Y + i * cols + b * V * 3;
        float2 acc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] = Yi[x * 3 + c];
        for (int mu = 0; mu < 4; ++mu) {
            const int64_t xp = shifted(g, co, mu, +1), xm = shifted(g, co, mu, -1);
            const double2 *u = U + (x * 4 + mu) * 9;
            const double2 *um = U + (xm * 4 + mu) * 9;
            const float2 *Yp = Yi + (1 + 2 * mu) * plane, *Ym = Yi + (2 + 2 * mu) * plane;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int bb = 0; bb < 3; ++bb) {
                    cfmac(acc[a], cvt<float2, double2>(um[bb * 3 + a]), Yp[xm * 3 + bb]);
                    cfma(acc[a], cvt<float2, double2>(u[a * 3 + bb]), Ym[xp * 3 + bb]);
                }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) gh[i * cols + xb * 3 + c] = acc[c];
    }
}

// ---------------------------------------------------------------------------
// gate and its derivative, per (row, site) colour triple
// ---------------------------------------------------------------------------
__global__ void gate_kernel(float2 *__restrict__ h, const float2 *__restrict__ a, int64_t n3) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n3; t += (int64_t)gridDim.x * blockDim.x) {
        float2 v[3];
        float q = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) { v[c] = a[t * 3 + c]; q += v[c].x * v[c].x + v[c].y * v[c].y; }
        const float f = q / (1.f + q);
#pragma unroll
        for (int c = 0; c < 3; ++c) h[t * 3 + c] = f * v[c];
    }
}

__global__ void gate_bwd_kernel(float2 *__restrict__ ga, const float2 *__restrict__ a, const float2 *__restrict__ gh,
                                int64_t n3) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n3; t += (int64_t)gridDim.x * blockDim.x) {
        float2 v[3], g[3];
        float q = 0.f, re = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[c] = a[t * 3 + c];
            g[c] = gh[t * 3 + c];
            q += v[c].x * v[c].x + v[c].y * v[c].y;
            re += v[c].x * g[c].x + v[c].y * g[c].y;
        }
        const float f = q / (1.f + q), w = 2.f * re / ((1.f + q) * (1.f + q));
#pragma unroll
        for (int c = 0; c < 3; ++c) ga[t * 3 + c] = make_float2(f * g[c].x + w * v[c].x, f * g[c].y + w * v[c].y);
    }
}

// ---------------------------------------------------------------------------
// head layout [(j*Ls + s)*4 + spin][x*3 + c]  <->  internal fine fields
// ---------------------------------------------------------------------------
// Output field f = j*B + b (output j of batch member b):
// dir = 0: v_f <- vh;  dir = 1: vh <- scale * v_f
__global__ void head_to_internal_kernel(float2 *__restrict__ v, float2 *__restrict__ vh, int nout, int Ls,
                                        int64_t V, int B, int dir, float scale = 1.f) {
    const int64_t nelem = V * 12 * Ls, total = nelem * nout * B, cols = (int64_t)B * V * 3;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = t / nelem, e = t - f * nelem;
        const int64_t j = f / B, b = f - j * B;
        const int s = (int)(e % Ls);
        const int64_t sc = e / Ls, x = sc / 12;
        const int comp = (int)(sc - x * 12);
        const int64_t hidx = ((j * Ls + s) * 4 + comp / 3) * cols + (b * V + x) * 3 + comp % 3;
        if (dir == 0) v[t] = vh[hidx];
        else vh[hidx] = make_float2(scale * v[t].x, scale * v[t].y);
    }
}

// refinement input: h0[(s*4 + spin)][(b*V + x)*3 + c] = v_b[(x*12 + spin*3 + c)*Ls + s]
__global__ void fields_to_input_kernel(float2 *__restrict__ h0, const double2 *__restrict__ v, int Ls, int64_t V,
                                       int B, double alpha) {
    const int64_t nelem = V * 12 * Ls, cols = (int64_t)B * V * 3;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nelem * B; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / nelem, e = t - b * nelem;
        const int s = (int)(e % Ls);
        const int64_t sc = e / Ls, x = sc / 12;
        const int comp = (int)(sc - x * 12);
        h0[((int64_t)s * 4 + comp / 3) * cols + (b * V + x) * 3 + comp % 3] =
            make_float2((float)(alpha * v[t].x), (float)(alpha * v[t].y));
    }
}

// out = oscale * out + in: the scaled head output plus the skip connection
__global__ void add_skip_kernel(float2 *__restrict__ out, const double2 *__restrict__ in, int64_t n, double oscale) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = out[i];
        const double2 b = in[i];
        out[i] = make_float2((float)(oscale * a.x + b.x), (float)(oscale * a.y + b.y));
    }
}

// Gamma = gamma_5 R_5 on internal fields: (Gamma v)(site, comp, s) =
// sign(comp) v(site, comp, Ls-1-s), sign + for spins 0, 1 and - for 2, 3.
__device__ __forceinline__ float2 gamma_of(const float2 *f, int64_t e, int Ls) {
    const int s = (int)(e % Ls);
    const int64_t sc = e / Ls;
    const int comp = (int)(sc % 12);
    const float2 w = f[sc * Ls + (Ls - 1 - s)];
    return comp < 6 ? w : make_float2(-w.x, -w.y);
}

// H[2j] = (1 + Gamma)/2 v_j,  H[2j+1] = (1 - Gamma)/2 v_j
__global__ void split_kernel(float2 *__restrict__ H, const float2 *__restrict__ v, int nout, int Ls, int64_t nelem) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nelem * nout;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / nelem, e = t - j * nelem;
        const float2 a = v[t], b = gamma_of(v + j * nelem, e, Ls);
        H[(2 * j) * nelem + e] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
        H[(2 * j + 1) * nelem + e] = make_float2(0.5f * (a.x - b.x), 0.5f * (a.y - b.y));
    }
}

// adjoint of split_kernel: gv_j = (1 + Gamma)/2 g_2j + (1 - Gamma)/2 g_2j+1
__global__ void split_adj_kernel(float2 *__restrict__ gv, const float2 *__restrict__ gH, int nout, int Ls,
                                 int64_t nelem) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nelem * nout;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / nelem, e = t - j * nelem;
        const float2 *g0 = gH + (2 * j) * nelem, *g1 = gH + (2 * j + 1) * nelem;
        const float2 a0 = g0[e], b0 = gamma_of(g0, e, Ls), a1 = g1[e], b1 = gamma_of(g1, e, Ls);
        gv[t] = make_float2(0.5f * (a0.x + b0.x + a1.x - b1.x), 0.5f * (a0.y + b0.y + a1.y - b1.y));
    }
}

// ---------------------------------------------------------------------------
// block-projection loss
// ---------------------------------------------------------------------------
struct NBlocks {
    int L[4], b[4], Lc[4];
    int run;          // elements per fine site = 12 * Ls
    int64_t bsites;   // sites per block
    int64_t nblk;     // blocks
};

__device__ __forceinline__ int64_t nblock_addr(const NBlocks &m, int64_t blk, int64_t e) {
    int64_t i = e / m.run;
    const int rem = (int)(e - i * m.run);
    int64_t t = blk;
    const int c0 = (int)(t % m.Lc[0]); t /= m.Lc[0];
    const int c1 = (int)(t % m.Lc[1]); t /= m.Lc[1];
    const int c2 = (int)(t % m.Lc[2]);
    const int c3 = (int)(t / m.Lc[2]);
    const int o0 = (int)(i % m.b[0]); i /= m.b[0];
    const int o1 = (int)(i % m.b[1]); i /= m.b[1];
    const int o2 = (int)(i % m.b[2]);
    const int o3 = (int)(i / m.b[2]);
    const int64_t site = (((int64_t)(c3 * m.b[3] + o3) * m.L[2] + (c2 * m.b[2] + o2)) * m.L[1] + (c1 * m.b[1] + o1)) *
                             m.L[0] + (c0 * m.b[0] + o0);
    return site * m.run + rem;
}

// Gp[split][blk][k][l] = sum over the split's share of block blk of
// conj(F_k(e)) F_l(e), nf <= 64 fields; FP32 products over chunks of 32
// elements, FP64 sums.
constexpr int GCH = 32, MAXF = 64, PPT = MAXF * MAXF / NT;
__global__ void __launch_bounds__(NT) block_gram_kernel(double2 *__restrict__ Gp, const float2 *__restrict__ F, int nf,
                                                        int64_t nelem, NBlocks m, int splits) {
    extern __shared__ float2 sF[];  // [nf][GCH]
    const int64_t blk = blockIdx.x;
    const int sp = blockIdx.y;
    const int64_t ne = m.bsites * m.run;
    const int64_t per = (ne + splits - 1) / splits;
    const int64_t e0 = sp * per, e1 = min(ne, e0 + per);
    const int np = nf * nf;
    double2 acc[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) acc[q] = make_double2(0, 0);
    for (int64_t c0 = e0; c0 < e1; c0 += GCH) {
        for (int j = threadIdx.x; j < nf * GCH; j += NT) {
            const int k = j / GCH, e = j - k * GCH;
            float2 v = make_float2(0.f, 0.f);
            if (c0 + e < e1) v = F[(int64_t)k * nelem + nblock_addr(m, blk, c0 + e)];
            sF[k * GCH + e] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const int p = threadIdx.x + q * NT;
            if (p < np) {
                const int k = p / nf, l = p - k * nf;
                float2 s = make_float2(0.f, 0.f);
#pragma unroll 8
                for (int e = 0; e < GCH; ++e) cfmac(s, sF[k * GCH + e], sF[l * GCH + e]);
                acc[q].x += (double)s.x;
                acc[q].y += (double)s.y;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int p = threadIdx.x + q * NT;
        if (p < np) Gp[((int64_t)sp * m.nblk + blk) * np + p] = acc[q];
    }
}

// Per block: G = H^+ H and A = H^+ Q from the full Gram matrix of F = [H; Q]
// (summed over the splits), Cholesky G = R^+ R, Y = G^-1 A.  One thread per
// block, FP64.  info[blk] = 0, or 1 when G is not positive definite.
constexpr int MAXH = 48, MAXT = 64;
__global__ void block_solve_kernel(float2 *__restrict__ Y, int *__restrict__ info, double2 *__restrict__ work,
                                   const double2 *__restrict__ Gp, int splits, int nh, int nt, int64_t nblk) {
    const int64_t blk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (blk >= nblk) return;
    const int nf = nh + nt, np = nf * nf;
    double2 *Rm = work + blk * (int64_t)(nh * nh + nh * nt);  // R (upper), then Z = R^-+ A
    double2 *Z = Rm + nh * nh;
    auto gf = [&](int k, int l) {
        double2 s = make_double2(0, 0);
        for (int z = 0; z < splits; ++z) s = s + Gp[((int64_t)z * nblk + blk) * np + k * nf + l];
        return s;
    };
    double gmax = 0;
    for (int k = 0; k < nh; ++k) gmax = fmax(gmax, gf(k, k).x);
    int bad = !(gmax > 0.0);
    for (int j = 0; j < nh && !bad; ++j) {
        double d = gf(j, j).x;
        for (int i = 0; i < j; ++i) d -= Rm[i * nh + j].x * Rm[i * nh + j].x + Rm[i * nh + j].y * Rm[i * nh + j].y;
        if (!(d > 1e-12 * gmax)) { bad = 1; break; }
        const double rd = sqrt(d);
        Rm[j * nh + j] = make_double2(rd, 0);
        for (int k = j + 1; k < nh; ++k) {
            double2 s = gf(j, k);
            for (int i = 0; i < j; ++i) s = s - cmulc(Rm[i * nh + j], Rm[i * nh + k]);
            Rm[j * nh + k] = make_double2(s.x / rd, s.y / rd);
        }
    }
    info[blk] = bad;
    if (bad) return;
    // R^+ Z = A (forward substitution), then R Y = Z (back substitution, in place)
    for (int c = 0; c < nt; ++c) {
        for (int i = 0; i < nh; ++i) {
            double2 s = gf(i, nh + c);
            for (int k = 0; k < i; ++k) s = s - cmulc(Rm[k * nh + i], Z[k * nt + c]);
            const double rd = Rm[i * nh + i].x;
            Z[i * nt + c] = make_double2(s.x / rd, s.y / rd);
        }
        for (int i = nh - 1; i >= 0; --i) {
            double2 s = Z[i * nt + c];
            for (int k = i + 1; k < nh; ++k) s = s - cmul(Rm[i * nh + k], Z[k * nt + c]);
            const double rd = Rm[i * nh + i].x;
            Z[i * nt + c] = make_double2(s.x / rd, s.y / rd);
            Y[(blk * nh + i) * nt + c] = make_float2((float)Z[i * nt + c].x, (float)Z[i * nt + c].y);
        }
    }
}

// R_c(e) = Q_c(e) - sum_k H_k(e) Y[k][c]; per-CTA partial sums of |R|^2
__global__ void __launch_bounds__(NT) residual_kernel(float2 *__restrict__ R, double *__restrict__ lpart,
                                                      const float2 *__restrict__ F, const float2 *__restrict__ Y, int nh,
                                                      int nt, int64_t nelem, NBlocks m, int splits) {
    extern __shared__ float2 sY[];  // [nh][nt]
    __shared__ double red[NT / 32];
    const int64_t blk = blockIdx.x;
    const int sp = blockIdx.y;
    for (int i = threadIdx.x; i < nh * nt; i += NT) sY[i] = Y[blk * nh * nt + i];
    __syncthreads();
    const int64_t ne = m.bsites * m.run;
    const int64_t per = (ne + splits - 1) / splits;
    const int64_t e0 = sp * per, e1 = min(ne, e0 + per);
    const float2 *Q = F + (int64_t)nh * nelem;
    double acc = 0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += NT) {
        const int64_t ad = nblock_addr(m, blk, e);
        float2 hk[MAXH];
#pragma unroll
        for (int k = 0; k < MAXH; ++k)
            if (k < nh) hk[k] = F[(int64_t)k * nelem + ad];
        float part = 0.f;
        for (int c = 0; c < nt; ++c) {
            float2 r = Q[(int64_t)c * nelem + ad];
#pragma unroll
            for (int k = 0; k < MAXH; ++k)
                if (k < nh) {
                    const float2 y = sY[k * nt + c];
                    r.x -= hk[k].x * y.x - hk[k].y * y.y;
                    r.y -= hk[k].x * y.y + hk[k].y * y.x;
                }
            R[(int64_t)c * nelem + ad] = r;
            part += r.x * r.x + r.y * r.y;
        }
        acc += part;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < NT / 32; ++w) s += red[w];
        lpart[blk * splits + sp] = s;
    }
}

// gH_k(e) = -scale sum_c R_c(e) conj(Y[k][c]), written over H in F
__global__ void __launch_bounds__(NT) grad_h_kernel(float2 *__restrict__ F, const float2 *__restrict__ R,
                                                    const float2 *__restrict__ Y, int nh, int nt, int64_t nelem,
                                                    NBlocks m, int splits, float scale) {
    extern __shared__ float2 sY[];
    const int64_t blk = blockIdx.x;
    const int sp = blockIdx.y;
    for (int i = threadIdx.x; i < nh * nt; i += NT) sY[i] = Y[blk * nh * nt + i];
    __syncthreads();
    const int64_t ne = m.bsites * m.run;
    const int64_t per = (ne + splits - 1) / splits;
    const int64_t e0 = sp * per, e1 = min(ne, e0 + per);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += NT) {
        const int64_t ad = nblock_addr(m, blk, e);
        float2 rc[MAXT];
#pragma unroll
        for (int c = 0; c < MAXT; ++c)
            if (c < nt) rc[c] = R[(int64_t)c * nelem + ad];
        for (int k = 0; k < nh; ++k) {
            float2 g = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < MAXT; ++c)
                if (c < nt) {
                    const float2 y = sY[k * nt + c];  // R conj(Y)
                    g.x += rc[c].x * y.x + rc[c].y * y.y;
                    g.y += rc[c].y * y.x - rc[c].x * y.y;
                }
            F[(int64_t)k * nelem + ad] = make_float2(-scale * g.x, -scale * g.y);
        }
    }
}

__global__ void sum_kernel(double *__restrict__ out, const double *__restrict__ part, int64_t n, double scale) {
    __shared__ double red[NT / 32];
    double s = 0;
    for (int64_t i = threadIdx.x; i < n; i += NT) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < NT / 32; ++w) t += red[w];
        *out = t * scale;
    }
}

template <typename TO, typename TI>
__global__ void convert_kernel(TO *__restrict__ out, const TI *__restrict__ in, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = cvt<TO, TI>(in[i]);
}

// out = in rounded to BF16 (round to nearest even) and back: FP32 values
// that a BF16 weight store holds exactly
__global__ void round_bf16_kernel(float2 *__restrict__ out, const float2 *__restrict__ in, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = in[i];
        out[i] = make_float2(__bfloat162float(__float2bfloat16_rn(v.x)), __bfloat162float(__float2bfloat16_rn(v.y)));
    }
}

// Adam on (Re, Im) with the real gradient 2 (Re G, Im G)
__global__ void adam_kernel(float2 *__restrict__ P, const float2 *__restrict__ G, float2 *__restrict__ M1,
                            float2 *__restrict__ M2, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gr = 2.f * G[i].x, gi = 2.f * G[i].y;
        float2 m = M1[i], v = M2[i], p = P[i];
        m.x = b1 * m.x + (1.f - b1) * gr;
        m.y = b1 * m.y + (1.f - b1) * gi;
        v.x = b2 * v.x + (1.f - b2) * gr * gr;
        v.y = b2 * v.y + (1.f - b2) * gi * gi;
        p.x -= lr * (m.x / c1) / (sqrtf(v.x / c2) + eps);
        p.y -= lr * (m.y / c1) / (sqrtf(v.y / c2) + eps);
        M1[i] = m;
        M2[i] = v;
        P[i] = p;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int cin4(const dwf_net *net, int l) { return 4 * (l == 0 ? net->sh.c_in : net->sh.hidden); }

void gemm(dwf_net *net, dwf_ctx *c, float2 *C, const float2 *A, const float2 *B, int M, int N, int K, int64_t lda,
          int64_t ldb, int opA, int opB) {
    const int gx = (N + GBN - 1) / GBN, gy = (M + GBM - 1) / GBM;
    const int64_t tiles = (int64_t)gx * gy;
    int splits = 1;
    if (tiles < 2 * c->sm_count && K > 1024)
        splits = (int)std::min<int64_t>((2 * c->sm_count + tiles - 1) / tiles, K / 512);
    splits = std::max(1, std::min(splits, 64));
    int kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + GBK - 1) / GBK * GBK;
    splits = (K + kchunk - 1) / kchunk;
    if (splits <= 1) {
        cgemm_kernel<<<dim3(gx, gy, 1), 256, 0, c->stream>>>(C, A, B, M, N, K, lda, ldb, opA, opB, std::max(K, 1), 0);
        DWF_CHECK_LAUNCH();
        return;
    }
    const int64_t mn = (int64_t)M * N;
    const size_t need = sizeof(float2) * (size_t)mn * splits;
    if (net->gws.bytes < need) net->gws.alloc(need);
    cgemm_kernel<<<dim3(gx, gy, splits), 256, 0, c->stream>>>(net->gws.as<float2>(), A, B, M, N, K, lda, ldb, opA, opB,
                                                              kchunk, mn);
    DWF_CHECK_LAUNCH();
    sum_partials_kernel<<<grid1(c, mn), NT, 0, c->stream>>>(C, net->gws.as<float2>(), splits, mn);
    DWF_CHECK_LAUNCH();
}

void ensure_ws(dwf_net *net, dwf_ctx *c, int B) {
    DWF_REQUIRE(c->g.Ls == net->sh.Ls, DWF_EINVAL, "the network's Ls differs from the context's");
    int dev = 0;
    DWF_CUDA(cudaGetDevice(&dev));
    DWF_REQUIRE(dev == net->device, DWF_EINVAL, "the network lives on another device");
    if (net->V == c->g.V && net->B == B) return;
    const int64_t X3 = c->g.V * 3 * B;
    const int L = net->sh.layers, C4 = 4 * net->sh.hidden;
    net->h.clear();
    net->a.clear();
    net->S.clear();
    net->h.resize(L + 1);
    net->a.resize(L);
    net->S.resize(L);
    for (int l = 0; l <= L; ++l) net->h[l].alloc(sizeof(float2) * (l == 0 ? cin4(net, 0) : C4) * X3);
    for (int l = 0; l < L; ++l) {
        net->a[l].alloc(sizeof(float2) * C4 * X3);
        net->S[l].alloc(sizeof(float2) * 9 * cin4(net, l) * X3);
    }
    const int64_t nhead = (int64_t)net->sh.nout * net->sh.Ls * 4;
    net->vh.alloc(sizeof(float2) * nhead * X3);
    net->v.alloc(sizeof(float2) * nhead * X3);  // nout * B internal fields
    net->V = c->g.V;
    net->B = B;
    net->F.release();
    net->R.release();
    net->gh.release();
    net->ga.release();
    net->yt.release();
}

// layers and head on h[0] (already filled) for the current batch
// the weights a pass reads: FP32 masters (training), or their BF16 rounding
// for inference when the weight precision is BF16
const float2 *weights(dwf_net *net, dwf_ctx *c, bool infer) {
    if (!infer || net->wprec != DWF_BF16) return net->P.as<float2>();
    if (!net->pi_valid) {
        const int64_t n = net->nparams;
        if (net->Pi.bytes < sizeof(float2) * (size_t)n) net->Pi.alloc(sizeof(float2) * (size_t)n);
        round_bf16_kernel<<<grid1(c, n), NT, 0, c->stream>>>(net->Pi.as<float2>(), net->P.as<float2>(), n);
        DWF_CHECK_LAUNCH();
        net->pi_valid = true;
    }
    return net->Pi.as<float2>();
}

void forward_core(dwf_net *net, dwf_ctx *c, bool infer) {
    const float2 *Pw = weights(net, c, infer);
    const int64_t V = c->g.V, X3 = V * 3 * net->B;
    const int L = net->sh.layers, C4 = 4 * net->sh.hidden;
    const double2 *U = c->U64.as<double2>();
    for (int l = 0; l < L; ++l) {
        const int ci = cin4(net, l);
        transport_kernel<<<grid1(c, ci * V * net->B), NT, 0, c->stream>>>(net->S[l].as<float2>(),
                                                                          net->h[l].as<float2>(), U, c->g, ci, net->B);
        DWF_CHECK_LAUNCH();
        const float2 *W = Pw + net->off[l];
        gemm(net, c, net->a[l].as<float2>(), W, net->S[l].as<float2>(), C4, (int)X3, 9 * ci, 9 * ci, X3, 0, 0);
        gate_kernel<<<grid1(c, C4 * V * net->B), NT, 0, c->stream>>>(net->h[l + 1].as<float2>(), net->a[l].as<float2>(),
                                                                       (int64_t)C4 * V * net->B);
        DWF_CHECK_LAUNCH();
    }
    const int nhead = net->sh.nout * net->sh.Ls * 4;
    gemm(net, c, net->vh.as<float2>(), Pw + net->off[L], net->h[L].as<float2>(), nhead, (int)X3, C4, C4, X3, 0, 0);
    head_to_internal_kernel<<<grid1(c, (int64_t)nhead * X3), NT, 0, c->stream>>>(
        net->v.as<float2>(), net->vh.as<float2>(), net->sh.nout, net->sh.Ls, V, net->B, 0);
    DWF_CHECK_LAUNCH();
}

// the proposal from seeded (or given) noise
void forward_impl(dwf_net *net, dwf_ctx *c, const void *input, bool input_dev, unsigned seed, bool infer) {
    ensure_ws(net, c, 1);
    net->oscale = 1.f;
    const int64_t V = c->g.V, V3 = V * 3;
    const int64_t nin = (int64_t)cin4(net, 0) * V3;
    float2 *h0 = net->h[0].as<float2>();
    if (input) {
        const double2 *src = (const double2 *)input;
        if (!input_dev) {
            if (net->in64.bytes < sizeof(double2) * nin) net->in64.alloc(sizeof(double2) * nin);
            DWF_CUDA(cudaMemcpyAsync(net->in64.p, input, sizeof(double2) * nin, cudaMemcpyHostToDevice, c->stream));
            src = net->in64.as<double2>();
        }
        bcopy<float2, double2>(c, h0, src, nin);
    } else {
        if (net->in64.bytes < sizeof(double2) * nin) net->in64.alloc(sizeof(double2) * nin);
        gauss_fill<double2>(c, net->in64.as<double2>(), 1, nin, 1, V, false, seed, STREAM_NETWORK);
        bcopy<float2, double2>(c, h0, net->in64.as<double2>(), nin);
    }
    forward_core(net, c, infer);
}

// the refinement of B given internal FP64 fields: out_b = v_b + net(v_b)
void refine_impl(dwf_net *net, dwf_ctx *c, const double2 *fields, int B, bool infer) {
    DWF_REQUIRE(net->sh.c_in == net->sh.Ls && net->sh.nout == 1, DWF_EINVAL,
                "a refinement network needs c_in = Ls and nout = 1");
    DWF_REQUIRE(B >= 1, DWF_EINVAL, "no fields to refine");
    ensure_ws(net, c, B);
    const int64_t nelem = c->g.V * 12 * c->g.Ls;
    // unit-norm fields scaled to entries of order one, where the gate acts
    const double alpha = std::sqrt((double)nelem);
    net->oscale = (float)(1.0 / alpha);
    fields_to_input_kernel<<<grid1(c, nelem * B), NT, 0, c->stream>>>(net->h[0].as<float2>(), fields, c->g.Ls, c->g.V, B,
                                                                       alpha);
    DWF_CHECK_LAUNCH();
    forward_core(net, c, infer);
    add_skip_kernel<<<grid1(c, nelem * B), NT, 0, c->stream>>>(net->v.as<float2>(), fields, nelem * B, 1.0 / alpha);
    DWF_CHECK_LAUNCH();
}

double loss_grad_impl(dwf_net *net, dwf_ctx *c, const double2 *targets, int nt, const int block[4]) {
    const int64_t V = c->g.V, X3 = V * 3 * net->B;
    const int Ls = net->sh.Ls, nout = net->sh.nout * net->B, nh = 2 * nout, nf = nh + nt;
    const int64_t nelem = V * 12 * Ls;
    DWF_REQUIRE(nh <= MAXH, DWF_EINVAL, "at most 24 network outputs");
    DWF_REQUIRE(nt >= 1 && nt <= MAXT && nf <= MAXF, DWF_EINVAL, "target count out of range (outputs*2 + targets <= 64)");
    NBlocks m;
    m.nblk = 1;
    m.bsites = 1;
    for (int i = 0; i < 4; ++i) {
        DWF_REQUIRE(block[i] >= 1 && c->g.L[i] % block[i] == 0, DWF_EINVAL, "block must divide the lattice");
        m.L[i] = c->g.L[i];
        m.b[i] = block[i];
        m.Lc[i] = m.L[i] / m.b[i];
        m.nblk *= m.Lc[i];
        m.bsites *= m.b[i];
    }
    m.run = 12 * Ls;
    const size_t fbytes = sizeof(float2) * (size_t)nelem * nf;
    if (net->F.bytes < fbytes) net->F.alloc(fbytes);
    if (net->R.bytes < sizeof(float2) * (size_t)nelem * nt) net->R.alloc(sizeof(float2) * (size_t)nelem * nt);
    float2 *F = net->F.as<float2>();
    split_kernel<<<grid1(c, nelem * nout), NT, 0, c->stream>>>(F, net->v.as<float2>(), nout, Ls, nelem);
    DWF_CHECK_LAUNCH();
    bcopy<float2, double2>(c, F + (int64_t)nh * nelem, targets, nelem * nt);
    const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(64, (2 * c->sm_count + m.nblk - 1) / m.nblk));
    const size_t gp = sizeof(double2) * (size_t)splits * m.nblk * nf * nf;
    if (net->gpart.bytes < gp) net->gpart.alloc(gp);
    block_gram_kernel<<<dim3((unsigned)m.nblk, splits), NT, sizeof(float2) * nf * GCH, c->stream>>>(
        net->gpart.as<double2>(), F, nf, nelem, m, splits);
    DWF_CHECK_LAUNCH();
    const size_t yb = sizeof(float2) * (size_t)m.nblk * nh * nt;
    if (net->Y.bytes < yb) net->Y.alloc(yb);
    if (net->info.bytes < sizeof(int) * (size_t)m.nblk) net->info.alloc(sizeof(int) * m.nblk);
    const size_t wb = sizeof(double2) * (size_t)m.nblk * (nh * nh + nh * nt);
    if (net->gram.bytes < wb) net->gram.alloc(wb);
    block_solve_kernel<<<(unsigned)((m.nblk + 63) / 64), 64, 0, c->stream>>>(
        net->Y.as<float2>(), net->info.as<int>(), net->gram.as<double2>(), net->gpart.as<double2>(), splits, nh, nt,
        m.nblk);
    DWF_CHECK_LAUNCH();
    std::vector<int> info(m.nblk);
    DWF_CUDA(cudaMemcpyAsync(info.data(), net->info.p, sizeof(int) * m.nblk, cudaMemcpyDeviceToHost, c->stream));
    DWF_CUDA(cudaStreamSynchronize(c->stream));
    for (int v : info) DWF_REQUIRE(v == 0, DWF_EBREAKDOWN, "network outputs are linearly dependent on a block");
    const size_t lp = sizeof(double) * (size_t)m.nblk * splits;
    if (net->lpart.bytes < lp) net->lpart.alloc(lp);
    if (!net->lval.p) net->lval.alloc(sizeof(double));
    const size_t ysm = sizeof(float2) * nh * nt;
    residual_kernel<<<dim3((unsigned)m.nblk, splits), NT, ysm, c->stream>>>(
        net->R.as<float2>(), net->lpart.as<double>(), F, net->Y.as<float2>(), nh, nt, nelem, m, splits);
    DWF_CHECK_LAUNCH();
    const double scale = 1.0 / ((double)m.nblk * nt);
    sum_kernel<<<1, NT, 0, c->stream>>>(net->lval.as<double>(), net->lpart.as<double>(), m.nblk * splits, scale);
    DWF_CHECK_LAUNCH();
    grad_h_kernel<<<dim3((unsigned)m.nblk, splits), NT, ysm, c->stream>>>(F, net->R.as<float2>(), net->Y.as<float2>(),
                                                                          nh, nt, nelem, m, splits, (float)scale);
    DWF_CHECK_LAUNCH();
    // gradient through the split and the head layout
    float2 *gv = net->v.as<float2>();  // the outputs are no longer needed
    split_adj_kernel<<<grid1(c, nelem * nout), NT, 0, c->stream>>>(gv, F, nout, Ls, nelem);
    DWF_CHECK_LAUNCH();
    const int nhead = net->sh.nout * Ls * 4, C4 = 4 * net->sh.hidden, L = net->sh.layers;
    float2 *gvh = net->vh.as<float2>();
    head_to_internal_kernel<<<grid1(c, (int64_t)nhead * X3), NT, 0, c->stream>>>(gv, gvh, net->sh.nout, Ls, V, net->B,
                                                                                  1, net->oscale);
    DWF_CHECK_LAUNCH();
    float2 *Gr = net->G.as<float2>();
    // head: dHd = gvh h_L^+,  dh_L = Hd^+ gvh
    gemm(net, c, Gr + net->off[L], gvh, net->h[L].as<float2>(), nhead, C4, (int)X3, X3, X3, 0, 1);
    if (net->gh.bytes < sizeof(float2) * (size_t)C4 * X3) net->gh.alloc(sizeof(float2) * (size_t)C4 * X3);
    if (net->ga.bytes < sizeof(float2) * (size_t)C4 * X3) net->ga.alloc(sizeof(float2) * (size_t)C4 * X3);
    gemm(net, c, net->gh.as<float2>(), net->P.as<float2>() + net->off[L], gvh, C4, (int)X3, nhead, C4, X3, 1, 0);
    for (int l = L - 1; l >= 0; --l) {
        const int ci = cin4(net, l);
        gate_bwd_kernel<<<grid1(c, (int64_t)C4 * V * net->B), NT, 0, c->stream>>>(
            net->ga.as<float2>(), net->a[l].as<float2>(), net->gh.as<float2>(), (int64_t)C4 * V * net->B);
        DWF_CHECK_LAUNCH();
        // dW_l = ga S_l^+
        gemm(net, c, Gr + net->off[l], net->ga.as<float2>(), net->S[l].as<float2>(), C4, 9 * ci, (int)X3, X3, X3, 0, 1);
        if (l == 0) break;
        // dh_l = sum_d T_d^+ (W_l[d]^+ ga)
        const size_t yt = sizeof(float2) * (size_t)9 * ci * X3;
        if (net->yt.bytes < yt) net->yt.alloc(yt);
        gemm(net, c, net->yt.as<float2>(), net->P.as<float2>() + net->off[l], net->ga.as<float2>(), 9 * ci, (int)X3, C4,
             9 * ci, X3, 1, 0);
        transport_adj_kernel<<<grid1(c, (int64_t)ci * V * net->B), NT, 0, c->stream>>>(
            net->gh.as<float2>(), net->yt.as<float2>(), c->U64.as<double2>(), c->g, ci, net->B);
        DWF_CHECK_LAUNCH();
    }
    double loss = 0;
    DWF_CUDA(cudaMemcpyAsync(&loss, net->lval.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    DWF_CUDA(cudaStreamSynchronize(c->stream));
    net->have_grad = true;
    return loss;
}

}  // namespace

// ---- entry points used by api.cu ----
dwf_net *net_create_impl(dwf_ctx *c, const dwf_net_shape &s) {
    DWF_REQUIRE(s.c_in >= 1 && s.hidden >= 1 && s.layers >= 1 && s.nout >= 1 && s.Ls >= 1, DWF_EINVAL,
                "network shape fields must be >= 1");
    DWF_REQUIRE(s.layers <= 16 && s.hidden <= 256 && s.c_in <= 256 && 2 * s.nout <= MAXH, DWF_EINVAL,
                "network shape out of range");
    std::unique_ptr<dwf_net> net(new dwf_net);
    net->sh = s;
    DWF_CUDA(cudaGetDevice(&net->device));
    int64_t o = 0;
    for (int l = 0; l < s.layers; ++l) {
        net->off.push_back(o);
        o += (int64_t)4 * s.hidden * 9 * 4 * (l == 0 ? s.c_in : s.hidden);
    }
    net->off.push_back(o);
    o += (int64_t)s.nout * s.Ls * 4 * 4 * s.hidden;
    net->nparams = o;
    const size_t b = sizeof(float2) * (size_t)o;
    net->P.alloc(b);
    net->G.alloc(b);
    net->M1.alloc(b);
    net->M2.alloc(b);
    DWF_CUDA(cudaMemsetAsync(net->P.p, 0, b, c->stream));
    DWF_CUDA(cudaMemsetAsync(net->G.p, 0, b, c->stream));
    DWF_CUDA(cudaMemsetAsync(net->M1.p, 0, b, c->stream));
    DWF_CUDA(cudaMemsetAsync(net->M2.p, 0, b, c->stream));
    DWF_CUDA(cudaStreamSynchronize(c->stream));
    return net.release();
}

void net_set_params_impl(dwf_net *net, const void *p, bool dev) {
    const int64_t n = net->nparams;
    DevBuf tmp(sizeof(double2) * (size_t)n);
    DWF_CUDA(cudaMemcpy(tmp.p, p, sizeof(double2) * n, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    convert_kernel<float2, double2><<<(unsigned)std::min<int64_t>((n + NT - 1) / NT, 4096), NT>>>(
        net->P.as<float2>(), tmp.as<double2>(), n);
    DWF_CHECK_LAUNCH();
    DWF_CUDA(cudaMemset(net->M1.p, 0, net->M1.bytes));
    DWF_CUDA(cudaMemset(net->M2.p, 0, net->M2.bytes));
    DWF_CUDA(cudaDeviceSynchronize());
    net->adam_t = 0;
    net->have_grad = false;
    net->pi_valid = false;
}

void net_copy_out(dwf_net *net, const DevBuf &src, void *p, bool dev) {
    const int64_t n = net->nparams;
    DevBuf tmp(sizeof(double2) * (size_t)n);
    convert_kernel<double2, float2><<<(unsigned)std::min<int64_t>((n + NT - 1) / NT, 4096), NT>>>(
        tmp.as<double2>(), src.as<float2>(), n);
    DWF_CHECK_LAUNCH();
    DWF_CUDA(cudaDeviceSynchronize());
    DWF_CUDA(cudaMemcpy(p, tmp.p, sizeof(double2) * n, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
}

void net_get_params_impl(dwf_net *net, void *p, bool dev) { net_copy_out(net, net->P, p, dev); }

void net_forward_impl(dwf_net *net, dwf_ctx *c, const void *input, bool input_dev, unsigned seed, double2 *out) {
    forward_impl(net, c, input, input_dev, seed, true);
    unpack(c, out, net->v.p, DWF_F32, net->sh.nout);
    DWF_CUDA(cudaStreamSynchronize(c->stream));
}

void net_refine_impl(dwf_net *net, dwf_ctx *c, const double2 *fields, int B, double2 *out) {
    refine_impl(net, c, fields, B, true);
    unpack(c, out, net->v.p, DWF_F32, B);
    DWF_CUDA(cudaStreamSynchronize(c->stream));
}

double net_refine_loss_grad_impl(dwf_net *net, dwf_ctx *c, const double2 *fields, int B, const double2 *targets, int nt,
                                 const int block[4], void *grad, bool grad_dev) {
    refine_impl(net, c, fields, B, false);
    const double L = loss_grad_impl(net, c, targets, nt, block);
    if (grad) net_copy_out(net, net->G, grad, grad_dev);
    return L;
}

bool net_is_refiner(const dwf_net *net) { return net->sh.c_in == net->sh.Ls && net->sh.nout == 1; }

double net_loss_grad_impl(dwf_net *net, dwf_ctx *c, const void *input, bool input_dev, unsigned seed,
                          const double2 *targets, int nt, const int block[4], void *grad, bool grad_dev) {
    forward_impl(net, c, input, input_dev, seed, false);
    const double L = loss_grad_impl(net, c, targets, nt, block);
    if (grad) net_copy_out(net, net->G, grad, grad_dev);
    return L;
}

void net_adam_impl(dwf_net *net, double lr, double b1, double b2, double eps) {
    DWF_REQUIRE(net->have_grad, DWF_ESTATE, "net_adam needs a gradient from net_loss_grad");
    DWF_REQUIRE(lr > 0 && b1 >= 0 && b1 < 1 && b2 >= 0 && b2 < 1 && eps > 0, DWF_EINVAL, "bad Adam parameters");
    net->adam_t++;
    net->pi_valid = false;
    const float c1 = (float)(1.0 - std::pow(b1, net->adam_t)), c2 = (float)(1.0 - std::pow(b2, net->adam_t));
    const int64_t n = net->nparams;
    adam_kernel<<<(unsigned)std::min<int64_t>((n + NT - 1) / NT, 4096), NT>>>(
        net->P.as<float2>(), net->G.as<float2>(), net->M1.as<float2>(), net->M2.as<float2>(), n, (float)lr, (float)b1,
        (float)b2, (float)eps, c1, c2);
    DWF_CHECK_LAUNCH();
    DWF_CUDA(cudaDeviceSynchronize());
}

void net_set_wprec_impl(dwf_net *net, dwf_prec prec) {
    DWF_REQUIRE(prec == DWF_F32 || prec == DWF_BF16, DWF_EINVAL, "network weight precision must be F32 or BF16");
    net->wprec = prec;
    net->pi_valid = false;
}

long long net_nparams(const dwf_net *net) { return net->nparams; }
int net_nout(const dwf_net *net) { return net->sh.nout; }
void net_free(dwf_net *net) { delete net; }

}  // namespace dwf
