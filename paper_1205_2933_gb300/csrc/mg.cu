// Multigrid solver orchestration: the V-cycle (Sec. 2), its CGNR smoother,
// GCR on coarse levels (S2, recursing through the V-cycle of the next level),
// the adaptive setup (Sec. 2: Krylov iterations on A x = 0 from random
// vectors, optionally followed by inverse-iteration sweeps that replace each
// vector by an approximate solution of A x = v with the current multigrid)
// and the outer flexible GCR (Sec. 3) with FP64 true residuals at every
// restart.
//
// Precision: the V-cycle, its smoother and all inner Krylov vectors run in R
// (double for the plain method, float for the mixed one); coarse stencils use
// the link precision chosen per level; the outer solution and residual, the
// block Gram-Schmidt and the coarse-operator construction are FP64.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <cmath>

#include "mg.cuh"

namespace dwf {

static thread_local std::string g_last_error;
void set_last_error(const std::string &m) { g_last_error = m; }
const char *last_error() { return g_last_error.c_str(); }

namespace {

constexpr int SLOT_A = 0;  // scalar slots used by the solvers (double index)

// DWF_VERBOSE=1: per-cycle residual trace of the solvers on stderr
bool verbose() {
    static const bool v = [] {
        const char *e = getenv("DWF_VERBOSE");
        return e && atoi(e) != 0;
    }();
    return v;
}

template <typename R> DevBuf &Qbuf(Level &L);
template <> DevBuf &Qbuf<double>(Level &L) { return L.Q64; }
template <> DevBuf &Qbuf<float>(Level &L) { return L.Q32; }

template <typename R> std::vector<DevBuf> &wsv(MGState &mg, int l);
template <> std::vector<DevBuf> &wsv<double>(MGState &mg, int l) { return mg.ws64[l]; }
template <> std::vector<DevBuf> &wsv<float>(MGState &mg, int l) { return mg.ws32[l]; }

struct GcrInfo {
    int iters = 0;
    double rel = 0.0;
};

template <typename R> class Runner {
  public:
    using T = C<R>;
    dwf_ctx *c;
    MGState &mg;
    long long coarse_applies[MAX_LEVELS] = {0, 0, 0, 0};

    Runner(dwf_ctx *ctx, MGState &m) : c(ctx), mg(m) {}

    int64_t n(int l) const { return mg.lev[l].lg.nelem; }

    // workspace vector i of level l
    T *ws(int l, int i) {
        auto &v = wsv<R>(mg, l);
        if ((int)v.size() <= i) v.resize(i + 1);
        if (!v[i].p) v[i].alloc(sizeof(T) * n(l));
        return v[i].template as<T>();
    }

    T *Q(int l) { return Qbuf<R>(mg.lev[l]).template as<T>(); }

    void apply(int l, T *out, const T *in, bool dag) {
        if (l == 0) {
            dslash(c, out, in, dag, 1);
        } else {
            coarse_apply<R>(c, mg.lev[l], out, in, dag);
            coarse_applies[l]++;
        }
    }

    double norm2(int l, const T *x) {
        bnorm2<T>(c, SLOT_A, x, n(l));
        double v = read_scalar(c, SLOT_A);
        if (!std::isfinite(v)) throw Error{DWF_ENAN, "NaN or Inf in a norm"};
        return v;
    }
    double2 dot(int l, const T *x, const T *y) {
        bdot<T, T>(c, SLOT_A, x, y, n(l));
        double v[2];
        read_scalars(c, SLOT_A, 2, v);
        return make_double2(v[0], v[1]);
    }

    // nu CGNR iterations on A_l x = b.  x_zero: start from x = 0 (else from x).
    // b_zero: b = 0 (the adaptive setup's A x = 0).  The step coefficients
    // stay on the device: no host round trip inside the loop.
    // rtol > 0: also stop once |r| <= rtol |r_0| (tested every 8 iterations).
    void cgnr(int l, T *x, const T *b, int iters, bool x_zero, bool b_zero, double rtol = 0.0) {
        const int64_t N = n(l);
        T *r = ws(l, 0), *z = ws(l, 1), *p = ws(l, 2), *w = ws(l, 3);
        if (x_zero) {
            bzero<T>(c, x, N);
            if (b_zero) return;
            bcopy<T, T>(c, r, b, N);
        } else {
            apply(l, r, x, false);
            if (b_zero) rscale<T>(c, r, -1.0, N);
            else cxpay<T>(c, r, make_double2(-1.0, 0.0), b, N);  // r = b - A x
        }
        apply(l, z, r, true);
        bcopy<T, T>(c, p, z, N);
        const int S_ZZ0 = 64, S_ZZ1 = 65, S_WW = 66;
        int izz = S_ZZ0, inew = S_ZZ1;
        bnorm2<T>(c, izz, z, N);
        const int S_RR = 67;
        double r0 = 0.0;
        if (rtol > 0.0) {
            bnorm2<T>(c, S_RR, r, N);
            r0 = std::sqrt(read_scalar(c, S_RR));
        }
        // on the fine level the FP32 Dslash produces the norms of its outputs
        bool fused = false;
        if constexpr (std::is_same<R, float>::value) fused = (l == 0) && dslash_norm_fused(c);
        auto anorm = [&](T *out, const T *in, bool dag, int slot) {
            if constexpr (std::is_same<R, float>::value)
                if (fused) {
                    dslash_norm(c, out, in, dag, 1, slot, 0);
                    return;
                }
            apply(l, out, in, dag);
            bnorm2<T>(c, slot, out, N);
        };
        for (int it = 0; it < iters; ++it) {
            anorm(w, p, false, S_WW);
            cg_xr<T>(c, x, r, p, w, izz, S_WW, N);
            if (it + 1 == iters) break;
            if (rtol > 0.0 && (it + 1) % 8 == 0) {
                bnorm2<T>(c, S_RR, r, N);
                if (std::sqrt(read_scalar(c, S_RR)) <= rtol * r0) break;
            }
            anorm(z, r, true, inew);
            cg_p<T>(c, p, z, inew, izz, N);
            std::swap(izz, inew);
        }
    }

    // Flexible GCR on level l, right-preconditioned by the V-cycle of level l
    // when pc is set.  The directions w_k = A z_k are orthonormalised by
    // classical Gram-Schmidt (a second pass only when the first removed more
    // than 3/4 of |w|^2); the preconditioned vectors z_k are kept raw and the
    // triangular Gram-Schmidt transform T is kept on the host, so that the
    // solution update x += sum_k alpha_k T^-1 z is one pass per cycle.  This
    // spans the same directions as the oracle's modified Gram-Schmidt GCR.
    GcrInfo gcr(int l, T *x, const T *b, double tol, int maxit, int restart, bool pc, bool x_zero, bool b_zero) {
        const int64_t N = n(l);
        DWF_REQUIRE(restart >= 1 && restart <= MAX_RESTART + 1, DWF_EINVAL, "GCR restart out of range");
        T *r = ws(l, 10);
        std::vector<T *> Z(restart), W(restart);
        for (int i = 0; i < restart; ++i) {
            Z[i] = ws(l, 16 + i);
            W[i] = ws(l, 16 + restart + i);
        }
        double bnorm = b_zero ? 0.0 : std::sqrt(norm2(l, b));
        if (bnorm == 0.0) {
            if (x_zero) {
                bzero<T>(c, x, N);
                return GcrInfo{0, 0.0};
            }
            bnorm = 1.0;  // A x = 0 from a nonzero start: absolute residual
        }
        auto residual = [&]() {
            if (x_zero) {
                bcopy<T, T>(c, r, b, N);
                x_zero = false;
                return;
            }
            apply(l, r, x, false);
            if (b_zero) rscale<T>(c, r, -1.0, N);
            else cxpay<T>(c, r, make_double2(-1.0, 0.0), b, N);
        };
        if (x_zero) bzero<T>(c, x, N);
        residual();
        double rn = std::sqrt(norm2(l, r));
        GcrInfo info;
        int k = 0;
        // host copy of the transform: Tm[i][j] (i <= j), and the step coefficients
        std::vector<double2> Tm((size_t)restart * restart), alpha(restart);
        auto finish_cycle = [&]() {
            if (k == 0) return;
            // gamma = T^-1 alpha (back substitution), x += sum_j gamma_j z_j
            std::vector<double2> g(k);
            for (int i = k - 1; i >= 0; --i) {
                double2 s = alpha[i];
                for (int j = i + 1; j < k; ++j) {
                    double2 t = cmul(Tm[(size_t)i * restart + j], g[j]);
                    s.x -= t.x;
                    s.y -= t.y;
                }
                double d = Tm[(size_t)i * restart + i].x;
                g[i] = make_double2(s.x / d, s.y / d);
            }
            for (int j0 = 0; j0 < k; j0 += 32) {
                int kk = std::min(32, k - j0);
                multiaxpy<T>(c, x, g.data() + j0, Z.data() + j0, kk, N);
            }
        };
        const int S_G = 128, S_WW = 124, S_A = 126;  // scalar slots
        while (info.iters < maxit && rn > tol * bnorm) {
            if (pc) vcycle(l, Z[k], r);
            else bcopy<T, T>(c, Z[k], r, N);
            apply(l, W[k], Z[k], false);
            for (int i = 0; i <= k; ++i) Tm[(size_t)i * restart + k] = make_double2(0, 0);
            // <W_i, W_k> for i < k and |W_k|^2 (as <W_k, W_k>) in one pass
            for (int pass = 0; pass < 2; ++pass) {
                bmultidot<T>(c, S_G, W.data(), k + 1, W[k], N);
                if (k > 0) multiaxpy_dev<T>(c, W[k], W.data(), k, S_G, -1.0, N);
                std::vector<double> v(2 * (k + 1));
                read_scalars(c, S_G, 2 * (k + 1), v.data());
                double before = v[2 * k], removed = 0.0;
                for (int i = 0; i < k; ++i) {
                    Tm[(size_t)i * restart + k].x += v[2 * i];
                    Tm[(size_t)i * restart + k].y += v[2 * i + 1];
                    removed += v[2 * i] * v[2 * i] + v[2 * i + 1] * v[2 * i + 1];
                }
                if (!std::isfinite(before)) throw Error{DWF_ENAN, "NaN or Inf in GCR"};
                if (k == 0 || removed < 0.75 * before) break;  // orthogonal enough
            }
            bnorm2<T>(c, S_WW, W[k], N);
            bdot<T, T>(c, S_A, W[k], r, N);
            double s[4];
            read_scalars(c, S_WW, 4, s);  // |w|^2, (unused), <w, r>
            double ww = s[0];
            if (!std::isfinite(ww) || !std::isfinite(s[2])) throw Error{DWF_ENAN, "NaN or Inf in GCR"};
            if (!(ww > 0.0)) break;
            double nw = std::sqrt(ww);
            Tm[(size_t)k * restart + k] = make_double2(nw, 0.0);
            alpha[k] = make_double2(s[2] / nw, s[3] / nw);  // <w_unit, r>
            // w_k <- w_k / |w_k|;  r -= alpha_k w_k
            rscale<T>(c, W[k], 1.0 / nw, N);
            caxpy<T>(c, r, make_double2(-alpha[k].x, -alpha[k].y), W[k], N);
            double a2 = alpha[k].x * alpha[k].x + alpha[k].y * alpha[k].y;
            double r2 = rn * rn - a2;
            rn = r2 > 0 ? std::sqrt(r2) : 0.0;
            ++info.iters;
            ++k;
            if (k == restart || rn <= tol * bnorm || info.iters >= maxit) {
                finish_cycle();
                residual();
                rn = std::sqrt(norm2(l, r));
                k = 0;
            }
        }
        finish_cycle();
        info.rel = rn / bnorm;
        return info;
    }

    // One V-cycle for A_l x = b (Sec. 2):
    //   x1 = S1^nu1(A, b); b2 = R(b - A x1); x2 = S2(R A P, b2);
    //   b3 = b - A(P x2 + x1); x = x1 + P x2 + S3^nu3(A, b3)
    // With the squared coarsening (Sec. 4) the coarse problem is that of the
    // normal equations: b2 = R D^+ (b - A x1).
    void vcycle(int l, T *x, const T *b) {
        const int64_t N = n(l);
        Level &L = mg.lev[l];
        const mg_params &p = mg.p;
        T *res = ws(l, 4), *sm = ws(l, 5), *b3 = ws(l, 6);
        T *b2 = ws(l + 1, 8), *x2 = ws(l + 1, 9);
        const bool squared = (l == 0 && p.coarsen == 1);
        if (p.nu_pre > 0) {
            cgnr(l, x, b, p.nu_pre, true, false);
            apply(l, res, x, false);
            cxpay<T>(c, res, make_double2(-1.0, 0.0), b, N);  // b - A x1
            if (squared) {
                apply(l, sm, res, true);
                restrict_any(L, b2, sm, l);
            } else {
                restrict_any(L, b2, res, l);
            }
        } else if (squared) {
            apply(l, sm, b, true);
            restrict_any(L, b2, sm, l);
        } else {
            restrict_any(L, b2, b, l);
        }
        coarse_solve(l + 1, x2, b2);
        prolong_any(L, x, x2, l, p.nu_pre > 0);
        if (p.nu_post > 0) {
            apply(l, res, x, false);
            bcopy<T, T>(c, b3, b, N);
            caxpy<T>(c, b3, make_double2(-1.0, 0.0), res, N);
            cgnr(l, sm, b3, p.nu_post, true, false);
            caxpy<T>(c, x, make_double2(1.0, 0.0), sm, N);
        }
    }

    // transfers with the FP16 basis copy when there is one (FP32 V-cycle only)
    void restrict_any(const Level &L, T *cout, const T *fin, int l) {
        if constexpr (std::is_same<R, float>::value)
            if (L.Q16.p) return restrict_h(c, L, cout, fin, L.Q16.as<__half2>());
        restrict_<R>(c, L, cout, fin, Q(l));
    }
    void prolong_any(const Level &L, T *fout, const T *cin, int l, bool acc) {
        if constexpr (std::is_same<R, float>::value)
            if (L.Q16.p) return prolong_h(c, L, fout, cin, L.Q16.as<__half2>(), acc);
        prolong_<R>(c, L, fout, cin, Q(l), acc);
    }

    void coarse_solve(int l, T *x, const T *b) {
        const mg_params &p = mg.p;
        bool coarsest = (l == mg.nlevels - 1);
        Level &L = mg.lev[l];
        if (coarsest && coarse_gcr_fused_ok(L, p.coarse_restart)) {
            const int64_t N = n(l);
            const size_t zb = sizeof(T) * N * p.coarse_restart;
            if (L.cgZ.bytes < zb) { L.cgZ.alloc(zb); L.cgW.alloc(zb); }
            if (!L.cgPart.p) L.cgPart.alloc(coarse_gcr_part_bytes(c));
            if (!L.cgIters.p) {
                L.cgIters.alloc(sizeof(int));
                DWF_CUDA(cudaMemsetAsync(L.cgIters.p, 0, sizeof(int), c->stream));
            }
            coarse_gcr_fused<R>(c, L, x, b, ws(l, 10), L.cgZ.as<T>(), L.cgW.as<T>(), L.cgPart.as<double2>(),
                                L.cgIters.as<int>(), p.coarsest_tol, p.coarsest_maxiter, p.coarse_restart);
            return;
        }
        if (!coarsest && p.cycle == 1) {
            // W-cycle (Sec. 2): two V-cycles of this level, x = V(b); x += V(b - A x)
            const int64_t N = n(l);
            T *res = ws(l, 11), *t = ws(l, 12);
            vcycle(l, x, b);
            apply(l, res, x, false);
            cxpay<T>(c, res, make_double2(-1.0, 0.0), b, N);
            vcycle(l, t, res);
            caxpy<T>(c, x, make_double2(1.0, 0.0), t, N);
            return;
        }
        gcr(l, x, b, coarsest ? p.coarsest_tol : p.coarse_tol, coarsest ? p.coarsest_maxiter : p.coarse_maxiter,
            p.coarse_restart, !coarsest, true, false);
    }

    // iterations run by the fused coarsest solver since the last call (resets the counter)
    long long fused_iters(int l) {
        Level &L = mg.lev[l];
        if (!L.cgIters.p) return 0;
        int v = 0;
        DWF_CUDA(cudaMemcpyAsync(&v, L.cgIters.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        DWF_CUDA(cudaStreamSynchronize(c->stream));
        DWF_CUDA(cudaMemsetAsync(L.cgIters.p, 0, sizeof(int), c->stream));
        return v;
    }

    // normalise x (level l) and store it as FP64 into dst
    void store_normalised(int l, double2 *dst, const T *x) {
        double nn = std::sqrt(norm2(l, x));
        DWF_REQUIRE(nn > 0.0, DWF_EBREAKDOWN, "adaptive setup produced a zero vector");
        bcopy<double2, T>(c, dst, x, n(l));
        rscale<double2>(c, dst, 1.0 / nn, n(l));
    }

    // block Gram-Schmidt, basis copies and the coarse operator of level l+1
    // Gamma split, block Gram-Schmidt (FP64 accumulation) and the coarse
    // operator of level l+1, all from the basis in precision R.
    void build(int l) {
        Level &L = mg.lev[l];
        const int64_t N = n(l);
        gamma_split<R>(c, L, Q(l), L.vec64.as<double2>(), L.nadapt, mg.p.split != 0);
        if (!block_orthonormalise<R>(c, L, Q(l)))
            throw Error{DWF_EBREAKDOWN, "block Gram-Schmidt met linearly dependent near-null vectors"};
        DevBuf W(sizeof(T) * N * L.nv);
        if (mg.p.coarsen == 1) build_squared_coarse<R>(c, L, mg.lev[l + 1], Q(l), W.as<T>());
        else build_coarse_from<R>(c, L, mg.lev[l + 1], Q(l), W.as<T>());
        if (std::is_same<R, float>::value && mg.p.basis_prec == DWF_F16) {
            if (L.Q16.bytes < sizeof(__half2) * N * L.nv) L.Q16.alloc(sizeof(__half2) * N * L.nv);
            basis_to_half(c, L.Q16.as<__half2>(), L.Q32.as<float2>(), N * L.nv);
        } else {
            L.Q16.release();
        }
        mg.nlevels = l + 2;
        DWF_CUDA(cudaStreamSynchronize(c->stream));
    }

    void setup_level(int l, const void *start, bool start_on_host) {
        init_vectors(l, start, start_on_host);
        relax_vectors(l);
        finish_level(l);
    }

    // the random (or given) start vectors of level l into L.vec64
    void init_vectors(int l, const void *start, bool start_on_host) {
        Level &L = mg.lev[l];
        const mg_params &p = mg.p;
        const int64_t N = n(l);
        L.vec64.alloc(sizeof(double2) * N * L.nadapt);
        Qbuf<R>(L).alloc(sizeof(T) * N * L.nv);
        double2 *v = L.vec64.as<double2>();
        if (l == 0 && start) {
            DevBuf canon(sizeof(double2) * N * L.nadapt);
            DWF_CUDA(cudaMemcpyAsync(canon.p, start, canon.bytes,
                                     start_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
            pack(c, v, canon.as<double2>(), DWF_F64, L.nadapt);
            DWF_CUDA(cudaStreamSynchronize(c->stream));
        } else {
            gauss_fill<double2>(c, v, L.nadapt, N, L.lg.g.Ls, L.lg.g.V, l == 0, p.seed + (uint32_t)l, 4u);
        }
    }

    // CGNR on A x = 0 from each start vector, one vector at a time
    void relax_vectors(int l) {
        Level &L = mg.lev[l];
        const mg_params &p = mg.p;
        const int64_t N = n(l);
        double2 *v = L.vec64.as<double2>();
        T *xv = ws(l, 9);
        for (int j = 0; j < L.nadapt; ++j) {
            bcopy<T, double2>(c, xv, v + (int64_t)j * N, N);
            cgnr(l, xv, nullptr, p.setup_iters0, false, true, p.setup_tol0);
            store_normalised(l, v + (int64_t)j * N, xv);
        }
    }

    // global orthonormalisation, the coarse level, optional sweeps
    void finish_level(int l) {
        Level &L = mg.lev[l];
        const mg_params &p = mg.p;
        double2 *v = L.vec64.as<double2>();
        T *xv = ws(l, 9), *bv = ws(l, 8);
        orthonormalise_global(l, v, L.nadapt);
        build(l);
        const int64_t N = n(l);
        // inverse-iteration sweeps: v <- (approximate) A^-1 v with the current
        // multigrid-preconditioned GCR, then the set is re-orthonormalised
        for (int sw = 0; sw < p.setup_sweeps; ++sw) {
            for (int j = 0; j < L.nadapt; ++j) {
                bcopy<T, double2>(c, bv, v + (int64_t)j * N, N);
                gcr(l, xv, bv, p.setup_sweep_tol, p.setup_sweep_iters, p.setup_sweep_iters + 1, true, true, false);
                store_normalised(l, v + (int64_t)j * N, xv);
            }
            orthonormalise_global(l, v, L.nadapt);
            build(l);
        }
    }

    // Two passes of modified Gram-Schmidt over the whole set of FP64 vectors.
    void orthonormalise_global(int l, double2 *v, int nv) {
        const int64_t N = n(l);
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j < nv; ++j) {
                double2 *vj = v + (int64_t)j * N;
                for (int i = 0; i < j; ++i) {
                    bdot<double2, double2>(c, SLOT_A, v + (int64_t)i * N, vj, N);
                    double d[2];
                    read_scalars(c, SLOT_A, 2, d);
                    caxpy<double2>(c, vj, make_double2(-d[0], -d[1]), v + (int64_t)i * N, N);
                }
                bnorm2<double2>(c, SLOT_A, vj, N);
                double nn = std::sqrt(read_scalar(c, SLOT_A));
                DWF_REQUIRE(nn > 0.0 && std::isfinite(nn), DWF_EBREAKDOWN, "adaptive vectors became linearly dependent");
                rscale<double2>(c, vj, 1.0 / nn, N);
            }
    }

    // Outer flexible GCR in FP64: each cycle solves A e = r approximately with
    // up to `restart` V-cycle-preconditioned GCR iterations in precision R,
    // then x += e and r = b - D x is recomputed in FP64 (reliable update).
    dwf_status solve_one(double2 *b, double2 *x, double tol, mg_stats &st) {
        const mg_params &p = mg.p;
        const int64_t N = n(0);
        double2 *r64 = mg_ws64(0, 12), *t64 = mg_ws64(0, 13);
        bnorm2<double2>(c, SLOT_A, b, N);
        double bn = std::sqrt(read_scalar(c, SLOT_A));
        if (bn == 0.0) {
            bzero<double2>(c, x, N);
            st.true_res = 0.0;
            return DWF_OK;
        }
        auto true_residual = [&]() {
            dslash(c, t64, x, false, 1);
            bcopy<double2, double2>(c, r64, b, N);
            caxpy<double2>(c, r64, make_double2(-1.0, 0.0), t64, N);
            bnorm2<double2>(c, SLOT_A, r64, N);
            double v = read_scalar(c, SLOT_A);
            if (!std::isfinite(v)) throw Error{DWF_ENAN, "NaN or Inf in the residual"};
            return std::sqrt(v);
        };
        double rn = true_residual();
        int iters = 0;
        dwf_status status = DWF_OK;
        T *bR = ws(0, 8), *eR = ws(0, 9);
        const double floor_rel = std::is_same<R, float>::value ? 2e-6 : 0.0;
        while (rn > tol * bn) {
            if (iters >= p.outer_maxiter) {
                status = DWF_ENOCONV;
                break;
            }
            bcopy<T, double2>(c, bR, r64, N);
            double tin = std::max(tol * bn / rn, floor_rel);
            GcrInfo gi = gcr(0, eR, bR, tin, std::min(p.outer_restart, p.outer_maxiter - iters), p.outer_restart + 1,
                             true, true, false);
            if (gi.iters == 0) {
                status = DWF_EBREAKDOWN;
                break;
            }
            iters += gi.iters;
            st.restarts++;
            caxpy_mixed<double2, T>(c, x, make_double2(1.0, 0.0), eR, N);
            rn = true_residual();
            if (verbose()) fprintf(stderr, "[dwfmg] cycle %d iters %d |r|/|b| %.3e\n", st.restarts, gi.iters, rn / bn);
        }
        st.iters += iters;
        st.true_res = std::max(st.true_res, rn / bn);
        return status;
    }

    // The paper's comparison solver (Sec. 3): CG on the normal equations of
    // the fine operator in precision R.  Every `cycle` iterations a reliable
    // update folds the low-precision correction into the FP64 solution and
    // replaces the iterated residual by the FP64 true residual, keeping the
    // search direction (the Krylov recurrence is not restarted).
    dwf_status cgnr_solve_one(double2 *b, double2 *x, double tol, int maxiter, int cycle, mg_stats &st) {
        const int64_t N = n(0);
        double2 *r64 = mg_ws64(0, 12), *t64 = mg_ws64(0, 13);
        bnorm2<double2>(c, SLOT_A, b, N);
        double bn = std::sqrt(read_scalar(c, SLOT_A));
        if (bn == 0.0) {
            bzero<double2>(c, x, N);
            return DWF_OK;
        }
        auto true_residual = [&]() {
            dslash(c, t64, x, false, 1);
            bcopy<double2, double2>(c, r64, b, N);
            caxpy<double2>(c, r64, make_double2(-1.0, 0.0), t64, N);
            bnorm2<double2>(c, SLOT_A, r64, N);
            double v = read_scalar(c, SLOT_A);
            if (!std::isfinite(v)) throw Error{DWF_ENAN, "NaN or Inf in the residual"};
            return std::sqrt(v);
        };
        T *r = ws(0, 0), *z = ws(0, 1), *p = ws(0, 2), *w = ws(0, 3), *xr = ws(0, 9);
        const int S_ZZ0 = 64, S_ZZ1 = 65, S_WW = 66, S_RR = 67;
        double rn = true_residual();
        double r_last = rn;
        int iters = 0;
        bcopy<T, double2>(c, r, r64, N);
        bzero<T>(c, xr, N);
        apply(0, z, r, true);
        bcopy<T, T>(c, p, z, N);
        int izz = S_ZZ0, inew = S_ZZ1;
        bnorm2<T>(c, izz, z, N);
        while (rn > tol * bn && iters < maxiter) {
            apply(0, w, p, false);
            bnorm2<T>(c, S_WW, w, N);
            cg_xr<T>(c, xr, r, p, w, izz, S_WW, N);
            ++iters;
            bool reliable = (iters % cycle == 0);
            if (iters % 16 == 0 || reliable) {
                bnorm2<T>(c, S_RR, r, N);
                rn = std::sqrt(read_scalar(c, S_RR));
                // reliable update once the iterated residual fell by 10x since the last one
                if (rn < 0.1 * r_last) reliable = true;
            }
            if (reliable || rn <= tol * bn || iters >= maxiter) {
                caxpy_mixed<double2, T>(c, x, make_double2(1.0, 0.0), xr, N);
                bzero<T>(c, xr, N);
                rn = true_residual();
                r_last = rn;
                bcopy<T, double2>(c, r, r64, N);
                st.restarts++;
                if (rn <= tol * bn || iters >= maxiter) break;
            }
            apply(0, z, r, true);
            bnorm2<T>(c, inew, z, N);
            cg_p<T>(c, p, z, inew, izz, N);
            std::swap(izz, inew);
        }
        st.iters += iters;
        st.true_res = std::max(st.true_res, rn / bn);
        return rn <= tol * bn ? DWF_OK : DWF_ENOCONV;
    }

    double2 *mg_ws64(int l, int i) {
        auto &v = mg.ws64[l];
        if ((int)v.size() <= i) v.resize(i + 1);
        if (!v[i].p) v[i].alloc(sizeof(double2) * n(l));
        return v[i].as<double2>();
    }
};

// Batched solve: all right-hand sides advance together.  Fine-level kernels
// run over the whole batch (the Dslash with nrhs in its grid, the basis of
// the transfers read once per 12 right-hand sides); every right-hand side
// keeps its own GCR coefficients, triangular transform and convergence
// state, and stops changing once converged.  Coarsest-level solves run per
// right-hand side through the fused kernel.  FP32 V-cycle, 2 levels, nu_1 = 0.
template <typename R> class BatchRunner {
  public:
    using T = C<R>;
    dwf_ctx *c;
    MGState &mg;
    int nr;
    Runner<R> one;
    static constexpr int SB = 1024, SS = 160;  // per-RHS scalar slot blocks: SB + r*SS
    DevBuf dcoef;                              // per-RHS coefficient arrays (device)

    BatchRunner(dwf_ctx *ctx, MGState &m, int nrhs) : c(ctx), mg(m), nr(nrhs), one(ctx, m) {
        DWF_REQUIRE(SB + nr * SS <= NSCALAR, DWF_EINVAL, "too many right-hand sides in one batch");
        mg.bscratch.ensure(nr);
        dcoef.alloc(sizeof(double2) * (size_t)nr * (MAX_RESTART + 2));
        dscale.alloc(sizeof(double) * (size_t)nr);
    }

    int64_t n(int l) const { return mg.lev[l].lg.nelem; }

    T *wsb(int l, int i) {
        auto &v = mg.wsb[l];
        if ((int)v.size() <= i) v.resize(i + 1);
        const size_t bytes = sizeof(T) * (size_t)n(l) * nr;
        if (v[i].bytes < bytes) v[i].alloc(bytes);
        return v[i].template as<T>();
    }

    // the per-RHS scalar blocks SB + r*SS .. + SS, one synchronisation
    void read_block(std::vector<double> &out) {
        out.resize((size_t)nr * SS);
        DWF_CUDA(cudaMemcpyAsync(c->hscal, c->scal.as<double>() + SB, sizeof(double) * (size_t)nr * SS,
                                 cudaMemcpyDeviceToHost, c->stream));
        DWF_CUDA(cudaStreamSynchronize(c->stream));
        std::copy(c->hscal, c->hscal + (size_t)nr * SS, out.begin());
    }

    // The setup's relaxation for all nr start vectors v (FP64, level 0) at
    // once: CGNR on D x = 0 from x0 = v is CGNR on D e = -D x0 from e = 0
    // with x = x0 + e (the same iterates); a vector stops counting once |D x|
    // fell by rtol (checked every 8 iterations); the run ends when all have.
    void relax(double2 *v, int iters, double rtol) {
        const int64_t N = n(0), NT = N * nr;
        T *x0 = wsb(0, 8), *e = wsb(0, 9), *bb = wsb(0, 10);
        bcopy<T, double2>(c, x0, v, NT);
        dslash(c, bb, x0, false, nr);
        rscale<T>(c, bb, -1.0, NT);
        cgnr_b(e, bb, iters, rtol);
        caxpy<T>(c, x0, make_double2(1.0, 0.0), e, NT);
        for (int r = 0; r < nr; ++r) one.store_normalised(0, v + (size_t)r * N, x0 + (size_t)r * N);
    }

    // nu CGNR iterations on D x = b for every right-hand side from x = 0
    // (accumulate: added to what x holds); with rtol > 0 the iteration also
    // ends once every |r| fell by rtol (tested every 8 iterations).  Nothing
    // is copied: the first residual is b itself, the first direction is the
    // first z (kept in the other of two z buffers), and x is first written,
    // not read, unless it accumulates.
    // how many solution updates the smoother may defer: CG_MAXDEFER when two
    // more direction buffers per right-hand side fit (decided once per runner)
    int defer_ = 0;
    int max_defer() {
        if (!defer_) {
            const size_t need = 2 * sizeof(T) * (size_t)n(0) * nr;
            size_t fr = 0, tot = 0;
            DWF_CUDA(cudaMemGetInfo(&fr, &tot));
            const auto &v = mg.wsb[0];
            const bool held = v.size() > 11 && v[7].bytes >= need / 2 && v[11].bytes >= need / 2;
            defer_ = (held || (double)need < 0.5 * (double)fr) ? CG_MAXDEFER : 1;
        }
        return defer_;
    }

    static constexpr int CHUNK = 8;  // iterations per chunk of a long CGNR run in the residual-keeping form

    // whether the smoother may keep its nu residuals (nu fields per right-hand
    // side at workspace indices 100 ..): decided once per runner and nu;
    // DWF_SMOOTHER_HISTORY=0 in the environment selects the other form
    int hist_nu_ = -1;
    bool hist_ok_ = false;
    bool keep_history(int nu) {
        if (nu != hist_nu_) {
            if (const char *e = getenv("DWF_SMOOTHER_HISTORY"); e && atoi(e) == 0) {
                hist_nu_ = nu;
                hist_ok_ = false;
                return false;
            }
            const size_t need = sizeof(T) * (size_t)n(0) * nr * (size_t)(nu + 1);
            size_t fr = 0, tot = 0;
            DWF_CUDA(cudaMemGetInfo(&fr, &tot));
            const auto &v = mg.wsb[0];
            bool held = (int)v.size() >= 100 + nu;
            for (int j = 0; held && j < nu; ++j) held = v[100 + j].bytes >= need / (nu + 1);
            hist_ok_ = held || (double)need < 0.5 * (double)fr;
            hist_nu_ = nu;
        }
        return hist_ok_;
    }

    void cgnr_b(T *x, const T *b, int iters, double rtol = 0.0, bool accumulate = false) {
        const int64_t N = n(0), NT = N * nr;
        if (iters <= 0) {
            if (!accumulate) bzero<T>(c, x, NT);
            return;
        }
        // the FP32 Dslash can produce the norms of its outputs in its epilogue
        bool fused = false;
        if constexpr (std::is_same<R, float>::value) fused = dslash_norm_fused(c);
        T *w = wsb(0, 3);
        if constexpr (std::is_same<R, float>::value) {
            if (fused && accumulate && rtol <= 0.0 && iters <= 32 && keep_history(iters)) {
                // The smoother's form when its residuals z_0 .. z_{nu-1} fit in
                // memory: no direction p and no per-iteration solution update.
                // w = D p follows w_{k+1} = D z_{k+1} + b_k w_k (p_{k+1} = z_{k+1}
                // + b_k p_k), applied in the D Dslash's epilogue as z's update is
                // in the D^+ one, and x gains sum_k a_k p_k = sum_j g_j z_j once
                // at the end (cg_combine_b).  |z_k|^2 and |w_k|^2 stay in slots
                // ZB + k and WB + k, from which that kernel forms the g_j.
                constexpr int ZB = 8, WB = 72;
                std::vector<T *> Zh(iters);
                for (int j = 0; j < iters; ++j) Zh[j] = wsb(0, 100 + j);
                T *wb[2] = {w, wsb(0, 13)};
                dslash_norm(c, Zh[0], b, true, nr, SB + ZB, SS);         // z_0 = D^+ r_0, r_0 = b
                dslash_norm(c, wb[0], Zh[0], false, nr, SB + WB, SS);    // w_0 = D p_0, p_0 = z_0
                for (int k = 0; k + 1 < iters; ++k) {
                    // z_{k+1} = z_k - a_k D^+ w_k, a_k = |z_k|^2 / |w_k|^2
                    dslash_zupdate(c, Zh[k + 1], wb[k & 1], Zh[k], nr, SB + ZB + k + 1, SS, SB + ZB + k, SB + WB + k);
                    // w_{k+1} = D z_{k+1} + b_k w_k, b_k = |z_{k+1}|^2 / |z_k|^2
                    dslash_wupdate(c, wb[(k + 1) & 1], Zh[k + 1], wb[k & 1], nr, SB + WB + k + 1, SS, SB + ZB + k + 1,
                                   SB + ZB + k);
                }
                cg_combine_b<T>(c, x, Zh.data(), iters, SB, SS, ZB, WB, N, nr);
                return;
            }
            if (fused && !accumulate && keep_history(CHUNK + 1)) {
                // A long run (the setup's relaxation) in the same form, in
                // chunks of CHUNK iterations: each keeps its residuals in a ring
                // of CHUNK + 1 buffers, and its end adds sum a_k p_k to x and
                // forms the next chunk's first direction from the chunk's first
                // one and those residuals (cg_chunk_b).  A residual test (every
                // chunk) computes b - D x itself.  Norms in slot rings of RS.
                constexpr int RS = 2 * CHUNK, ZB = 8, WB = 8 + RS;
                T *pp = wsb(0, 2);
                T *wb[2] = {w, wsb(0, 13)};
                std::vector<T *> ring(CHUNK + 1);
                for (int j = 0; j <= CHUNK; ++j) ring[j] = wsb(0, 100 + j);
                auto zptr = [&](int k) { return k == 0 ? pp : ring[k % (CHUNK + 1)]; };  // z_0 is p_0
                const int irr = 3;
                std::vector<double> r0(nr, 0.0), sv;
                if (rtol > 0.0) {
                    norm2_b<T>(c, mg.bscratch, SB + irr, SS, b, N, nr);
                    read_block(sv);
                    for (int q = 0; q < nr; ++q) r0[q] = std::sqrt(sv[(size_t)q * SS + irr]);
                }
                dslash_norm(c, pp, b, true, nr, SB + ZB, SS);       // p_0 = z_0 = D^+ b
                dslash_norm(c, wb[0], pp, false, nr, SB + WB, SS);  // w_0 = D p_0
                std::vector<T *> zc(CHUNK);
                for (int k0 = 0; k0 < iters;) {
                    const int k1 = std::min(k0 + CHUNK, iters), m = k1 - k0;
                    const bool last = k1 == iters;
                    for (int k = k0; k < (last ? k1 - 1 : k1); ++k) {
                        dslash_zupdate(c, zptr(k + 1), wb[k & 1], zptr(k), nr, SB + ZB + (k + 1) % RS, SS,
                                       SB + ZB + k % RS, SB + WB + k % RS);
                        dslash_wupdate(c, wb[(k + 1) & 1], zptr(k + 1), wb[k & 1], nr, SB + WB + (k + 1) % RS, SS,
                                       SB + ZB + (k + 1) % RS, SB + ZB + k % RS);
                    }
                    const int nz = last ? m - 1 : m;
                    for (int t = 1; t <= nz; ++t) zc[t - 1] = zptr(k0 + t);
                    cg_chunk_b<T>(c, x, pp, zc.data(), m, !last, k0 == 0, SB, SS, ZB, WB, k0, RS, N, nr);
                    k0 = k1;
                    if (rtol > 0.0 && !last) {
                        T *rt = wsb(0, 0);
                        dslash_residual(c, rt, x, b, nr);
                        norm2_b<T>(c, mg.bscratch, SB + irr, SS, rt, N, nr);
                        read_block(sv);
                        bool all = true;
                        for (int q = 0; q < nr; ++q) all &= std::sqrt(sv[(size_t)q * SS + irr]) <= rtol * r0[q];
                        if (all) break;
                    }
                }
                return;
            }
        }
        T *p = wsb(0, 2);
        T *zbuf[2] = {wsb(0, 1), wsb(0, 5)};
        int zi = 0;
        int izz = 0, inew = 1;
        const int iww = 2;
        auto dnorm = [&](T *out, const T *in, bool dag, int slot) {
            if constexpr (std::is_same<R, float>::value)
                if (fused) return dslash_norm(c, out, in, dag, nr, SB + slot, SS);
            dslash(c, out, in, dag, nr);
            norm2_b<T>(c, mg.bscratch, SB + slot, SS, out, N, nr);
        };
        dnorm(zbuf[0], b, true, izz);  // z_0 = D^+ r_0 with r_0 = b
        const T *rin = b, *pin = zbuf[0];
        bool xinit = !accumulate;
        const int irr = 3;
        std::vector<double> r0(nr, 0.0), sv;
        if (rtol > 0.0) {
            norm2_b<T>(c, mg.bscratch, SB + irr, SS, b, N, nr);
            read_block(sv);
            for (int q = 0; q < nr; ++q) r0[q] = std::sqrt(sv[(size_t)q * SS + irr]);
        }
        if constexpr (std::is_same<R, float>::value) {
            if (fused && !(accumulate && rtol > 0.0)) {
                // r itself is never needed: the normal-equations residual
                // z = D^+ r follows its own recursion z <- z - a D^+ w (the
                // same iterates in exact arithmetic), which the D^+ Dslash
                // applies in its epilogue.  x += a p is deferred for up to
                // CG_MAXDEFER iterations (their directions kept in buffers of
                // their own), so that up to four steps reach x in one pass.
                // Per iteration this streams w = D p, z (in, out), p (in, out)
                // and, on average, a quarter of x (in, out) and of the
                // deferred directions.  A residual test (every 8 iterations)
                // computes b - D x itself.
                // direction buffers: p and, where memory allows, CG_MAXDEFER more
                const int md = max_defer();
                std::vector<T *> pool = {p, wsb(0, 6)};
                if (md > 1) {
                    pool.push_back(wsb(0, 7));
                    pool.push_back(wsb(0, 11));
                }
                const int ia = 5;                // steps of the pending directions: slots ia, ia+1, ...
                std::vector<T *> pend;           // directions whose steps are not in x yet
                auto take = [&](const T *avoid) {  // a pool buffer that is neither pin nor pending
                    for (T *q : pool)
                        if (q != avoid && std::find(pend.begin(), pend.end(), q) == pend.end()) return q;
                    throw Error{DWF_ESTATE, "smoother: no free direction buffer"};
                };
                for (int it = 0; it < iters; ++it) {
                    dnorm(w, pin, false, iww);
                    const int np = (int)pend.size();
                    if (it + 1 == iters) {
                        if (np) cg_pxd_b<T>(c, x, nullptr, pin, pend.data(), np, nullptr, SB, SS, izz, iww, inew, ia, N,
                                            nr, 2);
                        else cg_px_b<T>(c, x, p, pin, nullptr, SB, SS, izz, iww, inew, N, nr, true, xinit);
                        break;
                    }
                    zi ^= 1;
                    dslash_zupdate(c, zbuf[zi], w, zbuf[zi ^ 1], nr, SB + inew, SS, SB + izz, SB + iww);
                    const bool test = rtol > 0.0 && (it + 1) % 8 == 0;
                    if (np && (np == md || test)) {
                        T *out = pend[0];
                        cg_pxd_b<T>(c, x, out, pin, pend.data(), np, zbuf[zi], SB, SS, izz, iww, inew, ia, N, nr, 1);
                        pend.clear();
                        pin = out;
                    } else if (it > 0 && !test) {
                        // pin (a pool buffer from it = 1 on) joins the pending
                        T *out = take(pin);
                        cg_pxd_b<T>(c, x, out, pin, pend.data(), np, zbuf[zi], SB, SS, izz, iww, inew, ia, N, nr, 0);
                        pend.push_back(const_cast<T *>(pin));
                        pin = out;
                    } else {
                        T *out = (it == 0) ? p : const_cast<T *>(pin);
                        cg_px_b<T>(c, x, out, pin, zbuf[zi], SB, SS, izz, iww, inew, N, nr, false, xinit);
                        pin = out;
                    }
                    xinit = false;
                    std::swap(izz, inew);
                    if (test) {
                        T *rt = wsb(0, 0);
                        dslash_residual(c, rt, x, b, nr);
                        norm2_b<T>(c, mg.bscratch, SB + irr, SS, rt, N, nr);
                        read_block(sv);
                        bool all = true;
                        for (int q = 0; q < nr; ++q) all &= std::sqrt(sv[(size_t)q * SS + irr]) <= rtol * r0[q];
                        if (all) break;
                    }
                }
                return;
            }
        }
        // x += a p is deferred into the direction update, so each iteration
        // reads r, w (residual) and x, p, z (solution and direction) once
        T *r = wsb(0, 0);
        for (int it = 0; it < iters; ++it) {
            dnorm(w, pin, false, iww);
            bool last = it + 1 == iters;
            if (!last) {
                cg_r_b<T>(c, r, rin, w, SB, SS, izz, iww, N, nr);
                rin = r;
                if (rtol > 0.0 && (it + 1) % 8 == 0) {
                    norm2_b<T>(c, mg.bscratch, SB + irr, SS, r, N, nr);
                    read_block(sv);
                    bool all = true;
                    for (int q = 0; q < nr; ++q) all &= std::sqrt(sv[(size_t)q * SS + irr]) <= rtol * r0[q];
                    last = all;
                }
            }
            if (last) {
                cg_px_b<T>(c, x, p, pin, nullptr, SB, SS, izz, iww, inew, N, nr, true, xinit);  // x += a p
                break;
            }
            zi ^= 1;
            dnorm(zbuf[zi], r, true, inew);
            cg_px_b<T>(c, x, p, pin, zbuf[zi], SB, SS, izz, iww, inew, N, nr, false, xinit);
            xinit = false;
            pin = p;
            std::swap(izz, inew);
        }
    }

    // Coarsest-level solves of every right-hand side.  One fused solve fills
    // about a third of the SMs, so NS of them run at a time on side streams
    // (each with its own scratch), joined back to the context stream.
    static constexpr int NS = 3;
    cudaStream_t side[NS] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[NS] = {nullptr, nullptr, nullptr};
    DevBuf cs_r[NS], cs_Z[NS], cs_W[NS], cs_part[NS];

    DevBuf cb_r, cb_Z, cb_W, cb_part;  // scratch of the batched coarsest solver

    void coarse_solves(T *x2, const T *b2, int64_t Nc) {
        Level &Lc = mg.lev[1];
        const mg_params &p = mg.p;
        static const bool batched = [] {
            const char *e = getenv("DWF_COARSE_BATCH");
            return !(e && atoi(e) == 0);
        }();
        if (batched && coarse_gcr_batch_ok(Lc, p.coarse_restart, std::min(nr, 16))) {
            // all right-hand sides through one cooperative launch (16 at a time)
            const int w = std::min(nr, 16);
            const size_t vb = sizeof(T) * (size_t)Nc * w;
            if (cb_r.bytes < vb) {
                cb_r.alloc(vb);
                cb_Z.alloc(vb * p.coarse_restart);
                cb_W.alloc(vb * p.coarse_restart);
            }
            if (!cb_part.p) cb_part.alloc(coarse_gcr_batch_part_bytes(c));
            if (!Lc.cgIters.p) {
                Lc.cgIters.alloc(sizeof(int));
                DWF_CUDA(cudaMemsetAsync(Lc.cgIters.p, 0, sizeof(int), c->stream));
            }
            for (int r0 = 0; r0 < nr; r0 += w) {
                const int nb = std::min(w, nr - r0);
                coarse_gcr_fused_batch<R>(c, Lc, x2 + (size_t)r0 * Nc, b2 + (size_t)r0 * Nc, nb, cb_r.as<T>(),
                                          cb_Z.as<T>(), cb_W.as<T>(), cb_part.as<double2>(), Lc.cgIters.as<int>(),
                                          p.coarsest_tol, p.coarsest_maxiter, p.coarse_restart);
            }
            return;
        }
        if (!coarse_gcr_fused_ok(Lc, p.coarse_restart)) {
            for (int r = 0; r < nr; ++r) one.coarse_solve(1, x2 + (size_t)r * Nc, b2 + (size_t)r * Nc);
            return;
        }
        if (!side[0]) {
            for (int i = 0; i < NS; ++i) {
                DWF_CUDA(cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking));
                DWF_CUDA(cudaEventCreateWithFlags(&ev_join[i], cudaEventDisableTiming));
                cs_r[i].alloc(sizeof(T) * Nc);
                cs_Z[i].alloc(sizeof(T) * Nc * p.coarse_restart);
                cs_W[i].alloc(sizeof(T) * Nc * p.coarse_restart);
                cs_part[i].alloc(coarse_gcr_part_bytes(c));
            }
            DWF_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
            if (!Lc.cgIters.p) {
                Lc.cgIters.alloc(sizeof(int));
                DWF_CUDA(cudaMemsetAsync(Lc.cgIters.p, 0, sizeof(int), c->stream));
            }
        }
        DWF_CUDA(cudaEventRecord(ev_fork, c->stream));
        cudaStream_t main = c->stream;
        for (int i = 0; i < NS; ++i) DWF_CUDA(cudaStreamWaitEvent(side[i], ev_fork, 0));
        for (int r = 0; r < nr; ++r) {
            const int i = r % NS;
            c->stream = side[i];
            coarse_gcr_fused<R>(c, Lc, x2 + (size_t)r * Nc, b2 + (size_t)r * Nc, cs_r[i].as<T>(), cs_Z[i].as<T>(),
                                cs_W[i].as<T>(), cs_part[i].as<double2>(), Lc.cgIters.as<int>(), p.coarsest_tol,
                                p.coarsest_maxiter, p.coarse_restart);
        }
        c->stream = main;
        for (int i = 0; i < NS; ++i) {
            DWF_CUDA(cudaEventRecord(ev_join[i], side[i]));
            DWF_CUDA(cudaStreamWaitEvent(main, ev_join[i], 0));
        }
    }

    ~BatchRunner() {
        if (side[0] || gstream) cudaStreamSynchronize(c->stream);
        for (auto &g : graphs) {
            cudaGraphExecDestroy(g.exec);
            for (auto &r : g.rec) {
                c->prof_pool.push_back(r.a);
                c->prof_pool.push_back(r.b);
            }
        }
        if (gstream) cudaStreamDestroy(gstream);
        if (g_fork) cudaEventDestroy(g_fork);
        if (g_join) cudaEventDestroy(g_join);
        for (int i = 0; i < NS; ++i) {
            if (side[i]) cudaStreamDestroy(side[i]);
            if (ev_join[i]) cudaEventDestroy(ev_join[i]);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
    }

    // The batched V-cycle as CUDA graphs: the V-cycle for one (output, input,
    // batch width) is captured at its first use and replayed afterwards, so
    // its ~80 launches (transfers, the coarsest solve, the smoother's Dslash
    // and vector kernels) leave the host as one.  A batch width is first run
    // without capture once: the coarsest solver's tuning runs, and every
    // workspace, side stream and scratch buffer is allocated there, outside
    // any capture.  Launches the event profiler brackets inside a graph are
    // timed after each replay from the graph's own events.
    struct VGraph {
        T *x;
        const T *b;
        int nr;
        cudaGraphExec_t exec;
        std::vector<ProfRecord> rec;
        long long a64, a32;        // fine applications the graph performs
        unsigned long long kernels; // kernels it launches
    };
    std::vector<VGraph> graphs;
    std::vector<int> eager_nr;  // batch widths already run without capture
    // graphs are captured and replayed on a stream of their own (capture is
    // not possible on the legacy default stream a caller may have given),
    // forked from and joined to the context's stream around every use
    cudaStream_t gstream = nullptr;
    cudaEvent_t g_fork = nullptr, g_join = nullptr;

    void graph_enter() {
        if (!gstream) {
            DWF_CUDA(cudaStreamCreateWithFlags(&gstream, cudaStreamNonBlocking));
            DWF_CUDA(cudaEventCreateWithFlags(&g_fork, cudaEventDisableTiming));
            DWF_CUDA(cudaEventCreateWithFlags(&g_join, cudaEventDisableTiming));
        }
        DWF_CUDA(cudaEventRecord(g_fork, c->stream));
        DWF_CUDA(cudaStreamWaitEvent(gstream, g_fork, 0));
    }
    void graph_leave(cudaStream_t main) {
        c->stream = main;
        DWF_CUDA(cudaEventRecord(g_join, gstream));
        DWF_CUDA(cudaStreamWaitEvent(main, g_join, 0));
    }

    void vcycle_b(T *x, const T *b) {
        if (!mg.p.graph || c->gate) return vcycle_body(x, b);
        for (auto &g : graphs)
            if (g.x == x && g.b == b && g.nr == nr) return replay(g);
        if (std::find(eager_nr.begin(), eager_nr.end(), nr) == eager_nr.end()) {
            eager_nr.push_back(nr);
            return vcycle_body(x, b);
        }
        VGraph g{x, b, nr, nullptr, {}, 0, 0, 0};
        cudaGraph_t graph = nullptr;
        const long long a64 = c->applies64, a32 = c->applies32;
        const unsigned long long k0 = launch_count();
        cudaStream_t main = c->stream;
        graph_enter();
        c->stream = gstream;
        DWF_CUDA(cudaStreamBeginCapture(gstream, cudaStreamCaptureModeThreadLocal));
        c->cap_rec = &g.rec;
        try {
            vcycle_body(x, b);
        } catch (...) {
            c->cap_rec = nullptr;
            cudaStreamEndCapture(gstream, &graph);
            if (graph) cudaGraphDestroy(graph);
            c->stream = main;
            throw;
        }
        c->cap_rec = nullptr;
        // the capture ran nothing: its counts are booked at every replay
        g.a64 = c->applies64 - a64;
        g.a32 = c->applies32 - a32;
        g.kernels = launch_count() - k0;
        c->applies64 = a64;
        c->applies32 = a32;
        cudaError_t e = cudaStreamEndCapture(gstream, &graph);
        c->stream = main;
        DWF_CUDA(e);
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        DWF_CUDA(e);
        graph_leave(main);
        graphs.push_back(std::move(g));
        replay(graphs.back());
    }

    void replay(VGraph &g) {
        cudaStream_t main = c->stream;
        graph_enter();
        DWF_CUDA(cudaGraphLaunch(g.exec, gstream));
        graph_leave(main);
        c->applies64 += g.a64;
        c->applies32 += g.a32;
        note_launches(g.kernels);
        if (c->prof && !g.rec.empty()) {
            DWF_CUDA(cudaStreamSynchronize(c->stream));
            for (const ProfRecord &r : g.rec) {
                float ms = 0.f;
                DWF_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
                c->prof_rec.push_back(ProfRecord{r.cls, nullptr, nullptr, r.units, ms});
            }
        }
    }

    // one V-cycle for every right-hand side (nu_1 = 0)
    void vcycle_body(T *x, const T *b) {
        Level &L = mg.lev[0];
        const int64_t N = n(0), NT = N * nr, Nc = n(1);
        T *res = wsb(0, 4);
        T *b2 = wsb(1, 8), *x2 = wsb(1, 9);
        restrict_batch<R>(c, L, b2, b, one.Q(0), nr);
        coarse_solves(x2, b2, Nc);
        prolong_batch<R>(c, L, x, x2, one.Q(0), nr, false);
        if (mg.p.nu_post > 0) {
            bool fused = false;
            if constexpr (std::is_same<R, float>::value) {
                fused = dslash_norm_fused(c);
                if (fused) dslash_residual(c, res, x, b, nr);  // res = b - A x in the Dslash epilogue
            }
            if (!fused) {
                dslash(c, res, x, false, nr);
                cxpay<T>(c, res, make_double2(-1.0, 0.0), b, NT);  // res = b - A x
            }
            cgnr_b(x, res, mg.p.nu_post, 0.0, true);  // x += S3(res)
        }
    }

    // One cycle (at most `restart` iterations) of lockstep flexible GCR on the
    // fine level for every right-hand side from x = 0, right-preconditioned by
    // vcycle_b.  tol[r] is relative to |b_r|; a right-hand side stops changing
    // once its residual estimate meets it (tol[r] >= 1: untouched).  Returns
    // the summed iterations of the active right-hand sides.
    long long gcr_b(T *x, const T *b, const std::vector<double> &tol, int restart) {
        const int64_t N = n(0), NT = N * nr;
        DWF_REQUIRE(restart >= 1 && restart <= 32, DWF_EINVAL, "batched GCR restart must be in 1..32");
        T *rr = wsb(0, 10);
        std::vector<T *> Z(restart), W(restart);
        for (int i = 0; i < restart; ++i) {
            Z[i] = wsb(0, 16 + i);
            W[i] = wsb(0, 16 + restart + i);
        }
        bzero<T>(c, x, NT);
        bcopy<T, T>(c, rr, b, NT);
        std::vector<double> sv;
        norm2_b<T>(c, mg.bscratch, SB, SS, b, N, nr);
        read_block(sv);
        std::vector<double> bn(nr), rn(nr);
        std::vector<char> act(nr);
        for (int r = 0; r < nr; ++r) {
            bn[r] = std::sqrt(sv[(size_t)r * SS]);
            rn[r] = bn[r];
            act[r] = bn[r] > 0.0 && tol[r] < 1.0;
        }
        auto any = [&]() { for (int r = 0; r < nr; ++r) if (act[r]) return true; return false; };
        std::vector<double2> Tm((size_t)nr * restart * restart), alpha((size_t)nr * restart);
        std::vector<double2> al(nr);
        std::vector<double> scr(nr);
        long long active_iters = 0;
        int k = 0;
        while (k < restart && any()) {
            vcycle_b(Z[k], rr);
            dslash(c, W[k], Z[k], false, nr);
            for (int r = 0; r < nr; ++r)
                for (int i = 0; i <= k; ++i) Tm[(size_t)r * restart * restart + i * restart + k] = make_double2(0, 0);
            // classical Gram-Schmidt of W_k against W_0 .. W_{k-1} (a second pass
            // where the first removed 3/4 or more of |W_k|^2)
            for (int pass = 0; pass < 2; ++pass) {
                multidot_b<T>(c, mg.bscratch, SB, SS, W.data(), k + 1, W[k], N, nr);
                if (k > 0) multiaxpy_b<T>(c, W[k], W.data(), k, SB, SS, -1.0, N, nr);
                read_block(sv);
                bool again = false;
                for (int r = 0; r < nr; ++r) {
                    const double *v = sv.data() + (size_t)r * SS;
                    double removed = 0.0;
                    for (int i = 0; i < k; ++i) {
                        Tm[(size_t)r * restart * restart + i * restart + k].x += v[2 * i];
                        Tm[(size_t)r * restart * restart + i * restart + k].y += v[2 * i + 1];
                        removed += v[2 * i] * v[2 * i] + v[2 * i + 1] * v[2 * i + 1];
                    }
                    if (!std::isfinite(v[2 * k])) throw Error{DWF_ENAN, "NaN or Inf in batched GCR"};
                    if (act[r] && k > 0 && removed >= 0.75 * v[2 * k]) again = true;
                }
                if (!again) break;
            }
            // |W_k|^2 and <W_k, r> per right-hand side
            norm2_b<T>(c, mg.bscratch, SB + 2, SS, W[k], N, nr);
            T *wk = W[k];
            multidot_b<T>(c, mg.bscratch, SB + 4, SS, &wk, 1, rr, N, nr);
            read_block(sv);
            for (int r = 0; r < nr; ++r) {
                const double *v = sv.data() + (size_t)r * SS;
                const double ww = v[2];
                double2 &Td = Tm[(size_t)r * restart * restart + k * restart + k];
                const bool ok = ww > 0.0 && std::isfinite(ww);
                scr[r] = ok ? 1.0 / std::sqrt(ww) : 0.0;
                if (act[r] && ok) {
                    const double nw = std::sqrt(ww);
                    Td = make_double2(nw, 0.0);
                    al[r] = make_double2(v[4] / nw, v[5] / nw);
                    const double r2 = rn[r] * rn[r] - (al[r].x * al[r].x + al[r].y * al[r].y);
                    rn[r] = r2 > 0 ? std::sqrt(r2) : 0.0;
                    ++active_iters;
                } else {
                    Td = make_double2(1.0, 0.0);
                    al[r] = make_double2(0.0, 0.0);
                }
                alpha[(size_t)r * restart + k] = al[r];
            }
            DWF_CUDA(cudaMemcpyAsync(dcoef.p, al.data(), sizeof(double2) * nr, cudaMemcpyHostToDevice, c->stream));
            DWF_CUDA(cudaMemcpyAsync(dscale.p, scr.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, c->stream));
            gcr_wr_b<T>(c, W[k], rr, dscale.as<double>(), dcoef.as<double2>(), N, nr);
            for (int r = 0; r < nr; ++r)
                if (act[r] && rn[r] <= tol[r] * bn[r]) act[r] = 0;
            ++k;
        }
        // x += sum_j gamma_j z_j with gamma = T^-1 alpha for every right-hand side
        if (k > 0) {
            std::vector<double2> g((size_t)nr * k);
            for (int r = 0; r < nr; ++r) {
                const double2 *Tr = Tm.data() + (size_t)r * restart * restart;
                const double2 *ar = alpha.data() + (size_t)r * restart;
                for (int i = k - 1; i >= 0; --i) {
                    double2 s = ar[i];
                    for (int j = i + 1; j < k; ++j) {
                        double2 t = cmul(Tr[i * restart + j], g[(size_t)r * k + j]);
                        s.x -= t.x;
                        s.y -= t.y;
                    }
                    const double d = Tr[i * restart + i].x;
                    g[(size_t)r * k + i] = make_double2(s.x / d, s.y / d);
                }
            }
            DWF_CUDA(cudaMemcpyAsync(dcoef.p, g.data(), sizeof(double2) * g.size(), cudaMemcpyHostToDevice, c->stream));
            combo_b<T>(c, x, Z.data(), k, dcoef.as<double2>(), N, nr);
        }
        return active_iters;
    }

    // outer flexible GCR in FP64 with reliable updates, all right-hand sides together
    // Right-hand sides that have converged leave the batch: each outer cycle
    // gathers the unconverged residuals into the first slots and runs the
    // lockstep GCR on that smaller batch.
    dwf_status solve(double2 *b, double2 *x, double tol, mg_stats &st) {
        const mg_params &p = mg.p;
        const int nfull = nr;
        const int64_t N = n(0), NT = N * nfull;
        double2 *r64 = mg_wsb64(0), *t64 = mg_wsb64(1);
        std::vector<double> sv;
        norm2_b<double2>(c, mg.bscratch, SB, SS, b, N, nfull);
        read_block(sv);
        std::vector<double> bn(nfull), rn(nfull);
        for (int r = 0; r < nfull; ++r) bn[r] = std::sqrt(sv[(size_t)r * SS]);
        std::vector<int> idx;  // unconverged right-hand sides
        auto true_residual = [&]() {
            const int na = (int)idx.size();
            if (na == nfull) {
                dslash(c, t64, x, false, nfull);
                bcopy<double2, double2>(c, r64, b, NT);
                caxpy<double2>(c, r64, make_double2(-1.0, 0.0), t64, NT);
                norm2_b<double2>(c, mg.bscratch, SB, SS, r64, N, nfull);
            } else {
                for (int r : idx) {
                    const size_t o = (size_t)r * N;
                    dslash(c, t64 + o, x + o, false, 1);
                    bcopy<double2, double2>(c, r64 + o, b + o, N);
                    caxpy<double2>(c, r64 + o, make_double2(-1.0, 0.0), t64 + o, N);
                    norm2_b<double2>(c, mg.bscratch, SB + r * SS, SS, r64 + o, N, 1);
                }
            }
            read_block(sv);
            for (int r : idx) {
                rn[r] = std::sqrt(sv[(size_t)r * SS]);
                if (!std::isfinite(rn[r])) throw Error{DWF_ENAN, "NaN or Inf in the residual"};
            }
        };
        for (int r = 0; r < nfull; ++r) {
            if (bn[r] == 0.0) bzero<double2>(c, x + (size_t)r * N, N);  // x = 0 solves D x = 0 exactly
            else idx.push_back(r);
        }
        for (int r = 0; r < nfull; ++r) rn[r] = 0.0;
        if (!idx.empty()) true_residual();
        T *bR = wsb(0, 8), *eR = wsb(0, 9);
        long long iters = 0;
        int cycles = 0;
        const double floor_rel = std::is_same<R, float>::value ? 2e-6 : 0.0;
        dwf_status status = DWF_OK;
        while (true) {
            idx.clear();
            for (int r = 0; r < nfull; ++r)
                if (rn[r] > tol * bn[r]) idx.push_back(r);
            const int na = (int)idx.size();
            if (na == 0) break;
            if (cycles * p.outer_restart >= p.outer_maxiter) {
                status = DWF_ENOCONV;
                break;
            }
            std::vector<double> tin(na);
            for (int k = 0; k < na; ++k) {
                const int r = idx[k];
                tin[k] = std::max(tol * bn[r] / rn[r], floor_rel);
                if (na < nfull) bcopy<T, double2>(c, bR + (size_t)k * N, r64 + (size_t)r * N, N);
            }
            if (na == nfull) bcopy<T, double2>(c, bR, r64, NT);
            nr = na;
            long long gi = 0;
            try {
                gi = gcr_b(eR, bR, tin, std::min(p.outer_restart, 32));
            } catch (...) {
                nr = nfull;
                throw;
            }
            nr = nfull;
            if (gi == 0) {
                status = DWF_EBREAKDOWN;
                break;
            }
            iters += gi;
            ++cycles;
            st.restarts++;
            if (na == nfull) caxpy_mixed<double2, T>(c, x, make_double2(1.0, 0.0), eR, NT);
            else
                for (int k = 0; k < na; ++k)
                    caxpy_mixed<double2, T>(c, x + (size_t)idx[k] * N, make_double2(1.0, 0.0), eR + (size_t)k * N, N);
            true_residual();
            if (verbose()) {
                fprintf(stderr, "[dwfmg batch] cycle %d batch %d iters %lld |r|/|b|:", cycles, na, gi);
                for (int r = 0; r < nfull; ++r) fprintf(stderr, " %.2e", bn[r] > 0 ? rn[r] / bn[r] : 0.0);
                fprintf(stderr, "\n");
            }
        }
        st.iters += (int)iters;
        for (int r = 0; r < nfull; ++r) st.true_res = std::max(st.true_res, bn[r] > 0 ? rn[r] / bn[r] : 0.0);
        return status;
    }

    double2 *mg_wsb64(int i) {
        auto &v = mg.wsb64;
        if ((int)v.size() <= i) v.resize(i + 1);
        const size_t bytes = sizeof(double2) * (size_t)n(0) * nr;
        if (v[i].bytes < bytes) v[i].alloc(bytes);
        return v[i].as<double2>();
    }

    DevBuf dscale;  // per-RHS real scale factors (device)
};

bool batch_on() {
    static const bool on = [] {
        const char *e = getenv("DWF_BATCH");
        return !(e && atoi(e) == 0);
    }();
    return on;
}

template <typename R> bool batch_eligible(const MGState &mg, int nrhs) {
    return std::is_same<R, float>::value && nrhs > 1 && batch_on() && mg.nlevels == 2 && mg.p.nu_pre == 0 &&
           mg.p.outer_restart <= 32 && mg.p.coarsen == 0;
}

// Right-hand sides per batch: at most 32, and no more than the free device
// memory holds (9 + 2 * restart fine fields in precision R and two FP64
// fields per right-hand side, counting the batch workspaces already held).
// 1 means: solve one at a time.
// The widest batch (at most 32, at most nrhs) whose fine-level workspaces fit
// in 90% of the free device memory.  A workspace already held is reused when
// it is large enough and replaced when it is not (the old one is freed
// first), so only the growth of each workspace the batch uses counts: the
// FP32 fields 0-5, 8-10 (smoother, V-cycle, setup relaxation) and, for a
// solve, the 2 x restart GCR directions from 16 on and the two FP64 fields.
template <typename R> int batch_width(const MGState &mg, int nrhs, bool solve) {
    const int64_t N = mg.lev[0].lg.nelem;
    const int restart = std::min(mg.p.outer_restart, 32);
    std::vector<int> used = {0, 1, 2, 3, 4, 5, 6, 8, 9, 10};  // 7 and 11 only where they fit (max_defer)
    if (solve)
        for (int i = 0; i < 2 * restart; ++i) used.push_back(16 + i);
    auto held = [&](const std::vector<DevBuf> &v, int i) { return i < (int)v.size() ? (double)v[i].bytes : 0.0; };
    auto growth = [&](int nb) {
        double g = 0;
        for (int i : used) g += std::max(0.0, (double)N * nb * sizeof(C<R>) - held(mg.wsb[0], i));
        if (solve)
            for (int i = 0; i < 2; ++i) g += std::max(0.0, (double)N * nb * sizeof(double2) - held(mg.wsb64, i));
        return g;
    };
    size_t fr = 0, tot = 0;
    DWF_CUDA(cudaMemGetInfo(&fr, &tot));
    int nb = std::min(32, nrhs);
    while (nb > 1 && growth(nb) > 0.9 * (double)fr) --nb;
    return nb;
}

template <typename R>
dwf_status setup_t(dwf_ctx *c, MGState &mg, int levels, const void *start, bool start_on_host) {
    Runner<R> run(c, mg);
    mg.nlevels = 1;
    for (int l = 0; l + 1 < levels; ++l) {
        const int na = mg.lev[l].nadapt;
        // the fine level's start vectors relax together in the FP32 V-cycle precision
        if (l == 0 && std::is_same<R, float>::value && batch_on() && na > 1 && na <= 32 &&
            batch_width<R>(mg, na, false) == std::min(na, 32)) {
            run.init_vectors(0, start, start_on_host);
            {
                BatchRunner<R> br(c, mg, na);
                br.relax(mg.lev[0].vec64.as<double2>(), mg.p.setup_iters0, mg.p.setup_tol0);
            }
            run.finish_level(0);
        } else {
            run.setup_level(l, start, start_on_host);
        }
    }
    return DWF_OK;
}

// The batched path covers FP32 V-cycles on two levels with nu_1 = 0;
// DWF_BATCH=0 in the environment turns it off.
template <typename R>
dwf_status solve_t(dwf_ctx *c, MGState &mg, double2 *b, double2 *x, double tol, int nrhs, mg_stats &st) {
    int width = batch_eligible<R>(mg, nrhs) ? batch_width<R>(mg, nrhs, true) : 1;
    if (batch_eligible<R>(mg, nrhs) && width < std::min(nrhs, 32) && !mg.wsb[0].empty()) {
        // memory-bound: the workspaces another width left (e.g. the setup's
        // relaxation of all start vectors) give way to the solve's own
        for (int l = 0; l < MAX_LEVELS; ++l) mg.wsb[l].clear();
        mg.wsb64.clear();
        width = batch_width<R>(mg, nrhs, true);
    }
    if (width > 1) {
        const int64_t N = mg.lev[0].lg.nelem;
        dwf_status worst = DWF_OK;
        long long c0 = 0;
        for (int r0 = 0; r0 < nrhs; r0 += width) {
            const int nb = std::min(width, nrhs - r0);
            BatchRunner<R> br(c, mg, nb);
            dwf_status s = br.solve(b + (size_t)r0 * N, x + (size_t)r0 * N, tol, st);
            if (s != DWF_OK && worst == DWF_OK) worst = s;
            c0 += br.one.fused_iters(1);
        }
        st.coarse_applies[1] += c0;
        return worst;
    }
    Runner<R> run(c, mg);
    dwf_status worst = DWF_OK;
    const int64_t N = mg.lev[0].lg.nelem;
    for (int r = 0; r < nrhs; ++r) {
        dwf_status s = run.solve_one(b + r * N, x + r * N, tol, st);
        if (s != DWF_OK && worst == DWF_OK) worst = s;
    }
    for (int l = 0; l < MAX_LEVELS; ++l) {
        long long f = (l < mg.nlevels) ? run.fused_iters(l) : 0;
        st.coarse_applies[l] += run.coarse_applies[l] + f;
    }
    return worst;
}

template <typename R>
dwf_status cgnr_t(dwf_ctx *c, MGState &mg, double2 *b, double2 *x, double tol, int maxiter, int nrhs, mg_stats &st) {
    Runner<R> run(c, mg);
    dwf_status worst = DWF_OK;
    const int64_t N = mg.lev[0].lg.nelem;
    for (int r = 0; r < nrhs; ++r) {
        dwf_status s = run.cgnr_solve_one(b + r * N, x + r * N, tol, maxiter, 200, st);
        if (s != DWF_OK && worst == DWF_OK) worst = s;
    }
    return worst;
}

bool nv_supported(int nv) {
    switch (nv) {
        case 2: case 4: case 6: case 8: case 12: case 16: case 24: case 32: return true;
        default: return false;
    }
}

}  // namespace

int mg_nlevels_minus1(dwf_ctx *c) { return c->mg ? c->mg->nlevels - 1 : 0; }

void mg_free(dwf_ctx *c) {
    delete c->mg;
    c->mg = nullptr;
}

dwf_status mg_setup_impl(dwf_ctx *c, int levels, const int *nvec, const int (*block)[4], const mg_params &p,
                         const void *start, bool start_on_host) {
    mg_free(c);
    DWF_REQUIRE(p.smoother_prec == DWF_F64 || p.smoother_prec == DWF_F32, DWF_EINVAL, "smoother_prec must be F64 or F32");
    DWF_REQUIRE(p.nu_post >= 0 && p.nu_pre >= 0 && p.coarse_restart >= 1 &&
                    p.outer_restart >= 1 && p.outer_restart <= MAX_RESTART && p.setup_sweep_iters >= 1 &&
                    p.setup_sweep_iters <= MAX_RESTART && p.coarse_restart <= MAX_RESTART,
                DWF_EINVAL, "iteration parameters out of range");
    MGState *mg = new MGState();
    mg->p = p;
    std::memset(&mg->stats, 0, sizeof(mg->stats));
    Level &L0 = mg->lev[0];
    L0.index = 0;
    L0.lg.g = c->g;
    L0.lg.ncomp = 12;
    L0.lg.nelem = c->g.V * 12 * c->g.Ls;
    for (int l = 0; l + 1 < levels; ++l) {
        Level &L = mg->lev[l];
        Level &Lc = mg->lev[l + 1];
        bool ok = nv_supported(nvec[l]) && (!p.split || nvec[l] % 2 == 0);
        for (int i = 0; i < 4; ++i) ok = ok && block[l][i] >= 1 && L.lg.g.L[i] % block[l][i] == 0;
        if (p.coarsen == 1) {
            ok = ok && levels == 2;
            for (int i = 0; i < 4; ++i) ok = ok && (block[l][i] >= 2 || L.lg.g.L[i] == 1);
        }
        if (!ok || (p.coarsen != 0 && p.coarsen != 1)) {
            delete mg;
            return DWF_EINVAL;
        }
        for (int i = 0; i < 4; ++i) L.block[i] = block[l][i];
        L.nv = nvec[l];
        L.nadapt = p.split ? nvec[l] / 2 : nvec[l];
        Lc.index = l + 1;
        Lc.lg.g.ap = 0;
        Lc.lg.g.Ls = 1;
        for (int i = 0; i < 4; ++i) Lc.lg.g.L[i] = L.lg.g.L[i] / block[l][i];
        Lc.lg.g.V = (int64_t)Lc.lg.g.L[0] * Lc.lg.g.L[1] * Lc.lg.g.L[2] * Lc.lg.g.L[3];
        Lc.lg.ncomp = nvec[l];
        Lc.lg.nelem = Lc.lg.g.V * nvec[l];
        dwf_prec yp = p.coarse_prec[l];
        Lc.yprec = (yp == DWF_F32 || yp == DWF_BF16 || yp == DWF_F16) ? yp : DWF_F64;
        // periodic neighbours of every coarse site, once (the coarse kernels
        // read them): the offsets of the stencil after the site itself
        Lc.npts = p.coarsen == 1 ? 33 : 9;
        int off[33][4];
        squared_offsets(off);  // its first 9 offsets are the 9-point stencil's
        const Geom &g = Lc.lg.g;
        const int nn = Lc.npts - 1;
        std::vector<int> tab((size_t)g.V * nn);
        for (int64_t site = 0; site < g.V; ++site) {
            int co[4];
            site_coords(g, site, co);
            for (int d = 1; d <= nn; ++d) {
                int cc[4];
                for (int mu = 0; mu < 4; ++mu) cc[mu] = (co[mu] + off[d][mu] + g.L[mu]) % g.L[mu];
                tab[(size_t)site * nn + d - 1] = (int)site_index(g, cc);
            }
        }
        try {
            Lc.nbr.alloc(sizeof(int) * tab.size());
            DWF_CUDA(cudaMemcpy(Lc.nbr.p, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice));
        } catch (...) {
            delete mg;
            throw;
        }
    }
    c->mg = mg;
    try {
        if (p.smoother_prec == DWF_F32) setup_t<float>(c, *mg, levels, start, start_on_host);
        else setup_t<double>(c, *mg, levels, start, start_on_host);
    } catch (...) {
        mg_free(c);
        throw;
    }
    return DWF_OK;
}

dwf_status mg_solve_impl(dwf_ctx *c, const void *b, void *x, double tol, int nrhs, mg_stats *stats, bool host) {
    if (!c->mg || c->mg->nlevels < 2) return DWF_ESTATE;
    MGState &mg = *c->mg;
    auto t0 = std::chrono::steady_clock::now();
    mg_stats st;
    std::memset(&st, 0, sizeof(st));
    long long a64 = c->applies64, a32 = c->applies32;
    const int64_t N = mg.lev[0].lg.nelem;
    DevBuf bd, xd;
    double2 *bp = (double2 *)b, *xp = (double2 *)x;
    if (host) {
        bd.alloc(sizeof(double2) * N * nrhs);
        xd.alloc(sizeof(double2) * N * nrhs);
        DWF_CUDA(cudaMemcpyAsync(bd.p, b, bd.bytes, cudaMemcpyDefault, c->stream));
        DWF_CUDA(cudaMemcpyAsync(xd.p, x, xd.bytes, cudaMemcpyDefault, c->stream));
        bp = bd.as<double2>();
        xp = xd.as<double2>();
    }
    dwf_status s = (mg.p.smoother_prec == DWF_F32) ? solve_t<float>(c, mg, bp, xp, tol, nrhs, st)
                                                   : solve_t<double>(c, mg, bp, xp, tol, nrhs, st);
    if (host) DWF_CUDA(cudaMemcpyAsync(x, xd.p, xd.bytes, cudaMemcpyDefault, c->stream));
    DWF_CUDA(cudaStreamSynchronize(c->stream));
    check_tc_timeout(c);
    st.fine_applies_f64 = c->applies64 - a64;
    st.fine_applies_f32 = c->applies32 - a32;
    st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = st;
    return s;
}

namespace {
MGState &need_mg(dwf_ctx *c, int level, int lo, int hi_excl) {
    DWF_REQUIRE(c->mg && c->mg->nlevels >= 2, DWF_ESTATE, "mg_setup has not completed");
    DWF_REQUIRE(level >= lo && level < hi_excl && level < c->mg->nlevels, DWF_EINVAL, "level out of range");
    return *c->mg;
}
}  // namespace

void mg_level_info_impl(dwf_ctx *c, int level, int dims[4], int *ncomp) {
    MGState &mg = need_mg(c, level, 0, MAX_LEVELS);
    for (int i = 0; i < 4; ++i) dims[i] = mg.lev[level].lg.g.L[i];
    *ncomp = mg.lev[level].lg.ncomp;
}

void mg_get_vectors_impl(dwf_ctx *c, int level, double2 *out) {
    MGState &mg = need_mg(c, level, 0, mg_nlevels_minus1(c));
    const Level &L = mg.lev[level];
    if (L.Q64.p)
        DWF_CUDA(cudaMemcpyAsync(out, L.Q64.p, sizeof(double2) * L.lg.nelem * L.nv, cudaMemcpyDeviceToDevice, c->stream));
    else
        bcopy<double2, float2>(c, out, L.Q32.as<float2>(), L.lg.nelem * L.nv);
}

void mg_get_coarse_links_impl(dwf_ctx *c, int level, double2 *out) {
    MGState &mg = need_mg(c, level, 1, MAX_LEVELS);
    const Level &L = mg.lev[level];
    DWF_CUDA(cudaMemcpyAsync(out, L.Y64.p, sizeof(double2) * L.lg.g.V * L.npts * L.lg.ncomp * L.lg.ncomp,
                             cudaMemcpyDeviceToDevice, c->stream));
}

void mg_restrict_impl(dwf_ctx *c, int level, double2 *cout, const double2 *fin) {
    MGState &mg = need_mg(c, level, 0, mg_nlevels_minus1(c));
    Level &L = mg.lev[level];
    if (L.Q64.p) {
        restrict_<double>(c, L, cout, fin, L.Q64.as<double2>());
        return;
    }
    const int64_t nf = L.lg.nelem, nc = mg.lev[level + 1].lg.nelem;
    DevBuf f32(sizeof(float2) * nf), c32(sizeof(float2) * nc);
    bcopy<float2, double2>(c, f32.as<float2>(), fin, nf);
    restrict_<float>(c, L, c32.as<float2>(), f32.as<float2>(), L.Q32.as<float2>());
    bcopy<double2, float2>(c, cout, c32.as<float2>(), nc);
    DWF_CUDA(cudaStreamSynchronize(c->stream));
}

void mg_prolong_impl(dwf_ctx *c, int level, double2 *fout, const double2 *cin) {
    MGState &mg = need_mg(c, level, 0, mg_nlevels_minus1(c));
    Level &L = mg.lev[level];
    if (L.Q64.p) {
        prolong_<double>(c, L, fout, cin, L.Q64.as<double2>(), false);
        return;
    }
    const int64_t nf = L.lg.nelem, nc = mg.lev[level + 1].lg.nelem;
    DevBuf f32(sizeof(float2) * nf), c32(sizeof(float2) * nc);
    bcopy<float2, double2>(c, c32.as<float2>(), cin, nc);
    prolong_<float>(c, L, f32.as<float2>(), c32.as<float2>(), L.Q32.as<float2>(), false);
    bcopy<double2, float2>(c, fout, f32.as<float2>(), nf);
    DWF_CUDA(cudaStreamSynchronize(c->stream));
}

void mg_coarse_apply_impl(dwf_ctx *c, int level, void *out, const void *in, bool dag, dwf_prec prec) {
    MGState &mg = need_mg(c, level, 1, MAX_LEVELS);
    DWF_REQUIRE(prec == DWF_F64 || prec == DWF_F32, DWF_EINVAL, "field precision must be F64 or F32");
    if (prec == DWF_F64) coarse_apply<double>(c, mg.lev[level], (double2 *)out, (const double2 *)in, dag);
    else coarse_apply<float>(c, mg.lev[level], (float2 *)out, (const float2 *)in, dag);
}

namespace {
template <typename R> void coarse_solve_t(dwf_ctx *c, MGState &mg, int level, void *x, const void *b) {
    Runner<R> run(c, mg);
    using T = C<R>;
    T *xl = run.ws(level, 9), *bl = run.ws(level, 8);
    const int64_t N = mg.lev[level].lg.nelem;
    DWF_CUDA(cudaMemcpyAsync(bl, b, sizeof(T) * N, cudaMemcpyDeviceToDevice, c->stream));
    run.coarse_solve(level, xl, bl);
    DWF_CUDA(cudaMemcpyAsync(x, xl, sizeof(T) * N, cudaMemcpyDeviceToDevice, c->stream));
    DWF_CUDA(cudaStreamSynchronize(c->stream));
}
template <typename R> void vcycle_t(dwf_ctx *c, MGState &mg, double2 *x, const double2 *b, int nrhs) {
    const int64_t N = mg.lev[0].lg.nelem;
    const int width = batch_eligible<R>(mg, nrhs) ? batch_width<R>(mg, nrhs, false) : 1;
    if (width > 1) {
        for (int r0 = 0; r0 < nrhs; r0 += width) {
            const int nb = std::min(width, nrhs - r0);
            BatchRunner<R> br(c, mg, nb);
            C<R> *bR = br.wsb(0, 8), *xR = br.wsb(0, 9);
            bcopy<C<R>, double2>(c, bR, b + (size_t)r0 * N, N * nb);
            br.vcycle_b(xR, bR);
            bcopy<double2, C<R>>(c, x + (size_t)r0 * N, xR, N * nb);
        }
    } else {
        Runner<R> run(c, mg);
        C<R> *bR = run.ws(0, 8), *xR = run.ws(0, 9);
        for (int r = 0; r < nrhs; ++r) {
            bcopy<C<R>, double2>(c, bR, b + (size_t)r * N, N);
            run.vcycle(0, xR, bR);
            bcopy<double2, C<R>>(c, x + (size_t)r * N, xR, N);
        }
    }
    DWF_CUDA(cudaStreamSynchronize(c->stream));
}
}  // namespace

void mg_coarse_solve_impl(dwf_ctx *c, int level, void *x, const void *b) {
    MGState &mg = need_mg(c, level, 1, MAX_LEVELS);
    DWF_REQUIRE(level == mg.nlevels - 1, DWF_EINVAL, "mg_coarse_solve runs on the coarsest level");
    if (mg.p.smoother_prec == DWF_F32) coarse_solve_t<float>(c, mg, level, x, b);
    else coarse_solve_t<double>(c, mg, level, x, b);
}

void mg_get_adaptive_impl(dwf_ctx *c, int level, double2 *out) {
    MGState &mg = need_mg(c, level, 0, mg_nlevels_minus1(c));
    const Level &L = mg.lev[level];
    DWF_CUDA(cudaMemcpyAsync(out, L.vec64.p, sizeof(double2) * (size_t)L.lg.nelem * L.nadapt, cudaMemcpyDeviceToDevice,
                             c->stream));
    DWF_CUDA(cudaStreamSynchronize(c->stream));
}

void mg_vcycle_impl(dwf_ctx *c, double2 *x, const double2 *b, int nrhs) {
    MGState &mg = need_mg(c, 0, 0, 1);
    if (mg.p.smoother_prec == DWF_F32) vcycle_t<float>(c, mg, x, b, nrhs);
    else vcycle_t<double>(c, mg, x, b, nrhs);
    DWF_CUDA(cudaStreamSynchronize(c->stream));
    check_tc_timeout(c);
}

dwf_status cg_solve_impl(dwf_ctx *c, const void *b, void *x, double tol, int maxiter, int nrhs, dwf_prec prec,
                         mg_stats *stats, bool host) {
    DWF_REQUIRE(prec == DWF_F64 || prec == DWF_F32, DWF_EINVAL, "CG precision must be F64 or F32");
    auto t0 = std::chrono::steady_clock::now();
    // the solver needs only level-0 workspaces: a private state when no setup exists
    MGState local;
    MGState *mg = c->mg;
    if (!mg) {
        mg = &local;
        Level &L0 = local.lev[0];
        L0.index = 0;
        L0.lg.g = c->g;
        L0.lg.ncomp = 12;
        L0.lg.nelem = c->g.V * 12 * c->g.Ls;
        local.nlevels = 1;
    }
    mg_stats st;
    std::memset(&st, 0, sizeof(st));
    long long a64 = c->applies64, a32 = c->applies32;
    const int64_t N = c->g.V * 12 * c->g.Ls;
    DevBuf bd, xd;
    double2 *bp = (double2 *)b, *xp = (double2 *)x;
    if (host) {
        bd.alloc(sizeof(double2) * N * nrhs);
        xd.alloc(sizeof(double2) * N * nrhs);
        DWF_CUDA(cudaMemcpyAsync(bd.p, b, bd.bytes, cudaMemcpyDefault, c->stream));
        DWF_CUDA(cudaMemcpyAsync(xd.p, x, xd.bytes, cudaMemcpyDefault, c->stream));
        bp = bd.as<double2>();
        xp = xd.as<double2>();
    }
    dwf_status s = (prec == DWF_F32) ? cgnr_t<float>(c, *mg, bp, xp, tol, maxiter, nrhs, st)
                                     : cgnr_t<double>(c, *mg, bp, xp, tol, maxiter, nrhs, st);
    if (host) DWF_CUDA(cudaMemcpyAsync(x, xd.p, xd.bytes, cudaMemcpyDefault, c->stream));
    DWF_CUDA(cudaStreamSynchronize(c->stream));
    st.fine_applies_f64 = c->applies64 - a64;
    st.fine_applies_f32 = c->applies32 - a32;
    st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = st;
    return s;
}

}  // namespace dwf
