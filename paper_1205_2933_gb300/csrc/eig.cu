// Low-mode diagnostic (Sec. 2, Fig. 1 of the paper judges a coarse space by
// how much of each low eigenmode it contains).
//
// The smallest eigenpairs of the Hermitian positive operator D^+ D by
// subspace iteration on its inverse, (D^+ D)^-1 = D^-1 Gamma D^-1 Gamma
// (D^+ = Gamma D Gamma, Gamma = gamma_5 R_5), with the multigrid solver for
// D^-1, and Rayleigh-Ritz on the iterated subspace (a small Hermitian
// eigenproblem, solved on the host by cyclic Jacobi rotations).  The share
// of a field v inside the coarse space is |P^+ v|^2 / |v|^2 (P has
// block-orthonormal columns, so P P^+ is the orthogonal projector).
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "mg.cuh"

namespace dwf {

namespace {

using cd = std::complex<double>;

// out_f = Gamma in_f: (Gamma v)(site, comp, s) = +-v(site, comp, Ls-1-s),
// + for spins 0, 1 and - for spins 2, 3
__global__ void gamma5r5_kernel(double2 *__restrict__ out, const double2 *__restrict__ in, int nf, int64_t nelem,
                                int Ls) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nelem * nf;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = t / nelem, e = t - f * nelem;
        const int s = (int)(e % Ls);
        const int64_t sc = e / Ls;
        const double2 w = in[f * nelem + sc * Ls + (Ls - 1 - s)];
        out[t] = (sc % 12) < 6 ? w : make_double2(-w.x, -w.y);
    }
}

void gamma5r5(dwf_ctx *c, double2 *out, const double2 *in, int nf, int64_t nelem) {
    const int64_t n = nelem * nf;
    gamma5r5_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 16), 256, 0, c->stream>>>(
        out, in, nf, nelem, c->g.Ls);
    DWF_CHECK_LAUNCH();
}

// Eigen-decomposition of a Hermitian n x n matrix A (row-major) by cyclic
// Jacobi rotations: each rotation first makes A_pq real with a phase, then
// removes it with a plane rotation of angle theta, tan 2 theta = 2|A_pq| /
// (A_pp - A_qq).  On return w holds the eigenvalues ascending and the
// columns of V the eigenvectors.
void herm_eig(int n, std::vector<cd> A, std::vector<double> &w, std::vector<cd> &V) {
    V.assign((size_t)n * n, cd(0, 0));
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    auto a = [&](int i, int j) -> cd & { return A[(size_t)i * n + j]; };
    double total = 0;
    for (const cd &x : A) total += std::norm(x);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += std::norm(a(p, q));
        if (off <= 1e-30 * total || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double r = std::abs(a(p, q));
                if (r <= 1e-300) continue;
                const cd ph = a(p, q) / r;  // e^{i phi}
                const double th = 0.5 * std::atan2(2.0 * r, a(p, p).real() - a(q, q).real());
                const double cs = std::cos(th), sn = std::sin(th);
                const cd e = std::conj(ph);  // e^{-i phi}
                // A <- A G with G = diag(1, e^{-i phi}) [[c, -s], [s, c]]
                for (int i = 0; i < n; ++i) {
                    const cd aip = a(i, p), aiq = a(i, q);
                    a(i, p) = cs * aip + sn * e * aiq;
                    a(i, q) = -sn * aip + cs * e * aiq;
                }
                // A <- G^+ A
                for (int j = 0; j < n; ++j) {
                    const cd apj = a(p, j), aqj = a(q, j);
                    a(p, j) = cs * apj + sn * ph * aqj;
                    a(q, j) = -sn * apj + cs * ph * aqj;
                }
                a(p, q) = 0.0;
                a(q, p) = 0.0;
                for (int i = 0; i < n; ++i) {
                    const cd vip = V[(size_t)i * n + p], viq = V[(size_t)i * n + q];
                    V[(size_t)i * n + p] = cs * vip + sn * e * viq;
                    V[(size_t)i * n + q] = -sn * vip + cs * e * viq;
                }
            }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return a(x, x).real() < a(y, y).real(); });
    std::vector<cd> Vs((size_t)n * n);
    w.resize(n);
    for (int j = 0; j < n; ++j) {
        w[j] = a(idx[j], idx[j]).real();
        for (int i = 0; i < n; ++i) Vs[(size_t)i * n + j] = V[(size_t)i * n + idx[j]];
    }
    V.swap(Vs);
}

constexpr int SLOT_E = 96;  // scalar slots used here

// modified Gram-Schmidt, twice, over k FP64 fields
void orthonormalise(dwf_ctx *c, double2 *v, int k, int64_t N) {
    for (int pass = 0; pass < 2; ++pass)
        for (int j = 0; j < k; ++j) {
            double2 *vj = v + (int64_t)j * N;
            for (int i = 0; i < j; ++i) {
                bdot<double2, double2>(c, SLOT_E, v + (int64_t)i * N, vj, N);
                double d[2];
                read_scalars(c, SLOT_E, 2, d);
                caxpy<double2>(c, vj, make_double2(-d[0], -d[1]), v + (int64_t)i * N, N);
            }
            bnorm2<double2>(c, SLOT_E, vj, N);
            const double nn = std::sqrt(read_scalar(c, SLOT_E));
            DWF_REQUIRE(nn > 0.0 && std::isfinite(nn), DWF_EBREAKDOWN, "subspace became linearly dependent");
            rscale<double2>(c, vj, 1.0 / nn, N);
        }
}

// out_j = sum_i C[i][j] in_i (k fields, C row-major k x k)
void combine(dwf_ctx *c, double2 *out, double2 *in, const std::vector<cd> &C, int k, int64_t N) {
    std::vector<double2 *> ptr(k);
    for (int i = 0; i < k; ++i) ptr[i] = in + (int64_t)i * N;
    std::vector<double2> beta(k);
    for (int j = 0; j < k; ++j) {
        double2 *oj = out + (int64_t)j * N;
        bzero<double2>(c, oj, N);
        for (int i = 0; i < k; ++i) beta[i] = make_double2(C[(size_t)i * k + j].real(), C[(size_t)i * k + j].imag());
        multiaxpy<double2>(c, oj, beta.data(), ptr.data(), k, N);
    }
}

}  // namespace

void lowest_modes_impl(dwf_ctx *c, int k, int max_iters, double tol, unsigned seed, double *evals, double2 *V,
                       double *resid, int *iters_done) {
    DWF_REQUIRE(c->mg && c->mg->nlevels >= 2, DWF_ESTATE, "the low-mode diagnostic needs a finished mg_setup");
    DWF_REQUIRE(k >= 1 && k <= 32 && max_iters >= 1 && tol > 0.0, DWF_EINVAL, "k in 1..32, max_iters >= 1, tol > 0");
    const int64_t N = c->g.V * 12 * c->g.Ls;
    DevBuf Wb(sizeof(double2) * (size_t)N * k), Xb(sizeof(double2) * (size_t)N * k), Ab(sizeof(double2) * (size_t)N * k);
    double2 *W = Wb.as<double2>(), *X = Xb.as<double2>(), *AV = Ab.as<double2>();
    gauss_fill<double2>(c, V, k, N, c->g.Ls, c->g.V, false, seed, 8u);
    orthonormalise(c, V, k, N);
    // inner solves: accurate enough that the iterated subspace is not limited by them
    const double stol = std::min(1e-3 * tol, 1e-9);
    std::vector<double> w(k), res(k, 1.0);
    int it = 0;
    for (; it < max_iters; ++it) {
        // X = D^-1 Gamma D^-1 Gamma V = (D^+ D)^-1 V
        gamma5r5(c, W, V, k, N);
        bzero<double2>(c, X, N * k);
        mg_stats st;
        dwf_status s = mg_solve_impl(c, W, X, stol, k, &st, false);
        DWF_REQUIRE(s == DWF_OK, s, "inner multigrid solve of the low-mode iteration failed");
        gamma5r5(c, W, X, k, N);
        bzero<double2>(c, X, N * k);
        s = mg_solve_impl(c, W, X, stol, k, &st, false);
        DWF_REQUIRE(s == DWF_OK, s, "inner multigrid solve of the low-mode iteration failed");
        orthonormalise(c, X, k, N);
        // Rayleigh-Ritz with A = D^+ D on span(X)
        dslash(c, W, X, false, k);
        dslash(c, AV, W, true, k);
        std::vector<cd> H((size_t)k * k);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                bdot<double2, double2>(c, SLOT_E, X + (int64_t)i * N, AV + (int64_t)j * N, N);
                double d[2];
                read_scalars(c, SLOT_E, 2, d);
                H[(size_t)i * k + j] = cd(d[0], d[1]);
            }
        for (int i = 0; i < k; ++i)
            for (int j = i + 1; j < k; ++j) {  // exact Hermitian symmetry
                const cd m = 0.5 * (H[(size_t)i * k + j] + std::conj(H[(size_t)j * k + i]));
                H[(size_t)i * k + j] = m;
                H[(size_t)j * k + i] = std::conj(m);
            }
        std::vector<cd> C;
        herm_eig(k, H, w, C);
        combine(c, V, X, C, k, N);   // Ritz vectors
        combine(c, W, AV, C, k, N);  // A times them
        double worst = 0;
        for (int j = 0; j < k; ++j) {
            double2 *wj = W + (int64_t)j * N;
            caxpy<double2>(c, wj, make_double2(-w[j], 0.0), V + (int64_t)j * N, N);
            bnorm2<double2>(c, SLOT_E, wj, N);
            res[j] = std::sqrt(read_scalar(c, SLOT_E)) / std::max(std::fabs(w[j]), 1e-300);
            worst = std::max(worst, res[j]);
        }
        if (worst <= tol) {
            ++it;
            break;
        }
    }
    for (int j = 0; j < k; ++j) {
        evals[j] = w[j];
        if (resid) resid[j] = res[j];
    }
    if (iters_done) *iters_done = it;
    DWF_CUDA(cudaStreamSynchronize(c->stream));
}

void coarse_overlap_impl(dwf_ctx *c, int level, const double2 *f, int nf, double *out) {
    DWF_REQUIRE(c->mg && c->mg->nlevels >= 2 && level >= 0 && level + 1 < c->mg->nlevels, DWF_EINVAL,
                "level must have a coarser level");
    const int64_t N = c->mg->lev[level].lg.nelem, Nc = c->mg->lev[level + 1].lg.nelem;
    DevBuf cb(sizeof(double2) * (size_t)Nc);
    for (int j = 0; j < nf; ++j) {
        const double2 *fj = f + (int64_t)j * N;
        mg_restrict_impl(c, level, cb.as<double2>(), fj);
        bnorm2<double2>(c, SLOT_E, cb.as<double2>(), Nc);
        const double pc = read_scalar(c, SLOT_E);
        bnorm2<double2>(c, SLOT_E, fj, N);
        const double ff = read_scalar(c, SLOT_E);
        DWF_REQUIRE(ff > 0.0, DWF_EINVAL, "zero field");
        out[j] = pc / ff;
    }
}

}  // namespace dwf
