// Multigrid internals: per-level data, transfer and coarse-operator kernels,
// solver entry points.
#pragma once

#include "dwf_internal.cuh"
#include "dwfnet.h"

namespace dwf {

void set_last_error(const std::string &m);
const char *last_error();

constexpr int MAX_LEVELS = 4;

// A field on one level: V sites x ncomp components x Ls (fine: ncomp = 12,
// Ls = Ls; coarse: ncomp = Nvec, Ls = 1), element (site*ncomp + comp)*Ls + s.
struct LevelGeom {
    Geom g;        // g.Ls = 1 on coarse levels
    int ncomp;     // components per site and s
    int64_t nelem; // complex elements per field
};

struct Level {
    int index = 0;         // 0 = fine lattice
    LevelGeom lg;
    // transfer to level + 1 (absent on the coarsest level)
    int block[4] = {1, 1, 1, 1};
    int nv = 0;            // coarse components per site of level + 1
    int nadapt = 0;        // adaptive vectors (nv / 2 when split)
    DevBuf Q64, Q32;       // nv block-orthonormalised fields of this level
    DevBuf Q16;            // FP16 copy used by the FP32 V-cycle's transfers (basis_prec = F16)
    DevBuf vec64;          // nadapt adaptive vectors (unsplit, normalised), FP64
    // coarse operator of this level (levels >= 1): [V][npts][n][n] complex,
    // npts = 9 for R A P, 33 for the squared operator's P^+ D^+ D P
    int npts = 9;
    DevBuf Y64, Y32, Y16;  // Y16 holds bf16 or fp16 pairs per coarse_prec
    DevBuf Ytc;            // BF16 stencil as per-site tensor-core operand images (coarse_gcr_tc.cu)
    dwf_prec yprec = DWF_F64;
    // block reductions scratch: [Vc][nv][nv] complex FP64
    DevBuf G, F, Rinv;
    DevBuf info;           // int per coarse site: Cholesky status
    // fused coarsest-level GCR: contiguous direction vectors, partial sums, counter
    DevBuf cgZ, cgW, cgPart, cgIters;
    // coarse levels: neighbour table int [V][npts - 1], entry 2 mu (+mu) and
    // 2 mu + 1 (-mu), then (33 points) the diagonals in stencil order
    DevBuf nbr;
};

// ---- blasb.cu ---- batched vector kernels: nrhs fields of n elements, per-RHS
// scalars at slot blocks base + r*stride of ctx->scal
struct BatchScratch {
    DevBuf part, count;
    void ensure(int nrhs);
};
struct MGState {
    int nlevels = 0;
    mg_params p;
    Level lev[MAX_LEVELS];
    // workspaces (allocated lazily by precision)
    std::vector<DevBuf> ws64[MAX_LEVELS], ws32[MAX_LEVELS];
    // batched solve: nrhs-wide workspaces and reduction scratch
    std::vector<DevBuf> wsb[MAX_LEVELS], wsb64;
    BatchScratch bscratch;
    mg_stats stats;
};

void mg_free(dwf_ctx *c);
int mg_nlevels_minus1(dwf_ctx *c);
dwf_status mg_setup_impl(dwf_ctx *c, int levels, const int *nvec, const int (*block)[4], const mg_params &p,
                         const void *start, bool start_on_host);
dwf_status mg_solve_impl(dwf_ctx *c, const void *b, void *x, double tol, int nrhs, mg_stats *stats, bool host);
dwf_status cg_solve_impl(dwf_ctx *c, const void *b, void *x, double tol, int maxiter, int nrhs, dwf_prec prec,
                         mg_stats *stats, bool host);
// component calls of the C ABI (see dwfmg.h); throw Error on bad arguments
void mg_level_info_impl(dwf_ctx *c, int level, int dims[4], int *ncomp);
void mg_get_vectors_impl(dwf_ctx *c, int level, double2 *out);
void mg_get_coarse_links_impl(dwf_ctx *c, int level, double2 *out);
void mg_restrict_impl(dwf_ctx *c, int level, double2 *cout, const double2 *fin);
void mg_prolong_impl(dwf_ctx *c, int level, double2 *fout, const double2 *cin);
void mg_coarse_apply_impl(dwf_ctx *c, int level, void *out, const void *in, bool dag, dwf_prec prec);
void mg_vcycle_impl(dwf_ctx *c, double2 *x, const double2 *b, int nrhs);
void mg_get_adaptive_impl(dwf_ctx *c, int level, double2 *out);
// ---- eig.cu ---- low-mode diagnostic
void lowest_modes_impl(dwf_ctx *c, int k, int max_iters, double tol, unsigned seed, double *evals, double2 *V,
                       double *resid, int *iters_done);
void coarse_overlap_impl(dwf_ctx *c, int level, const double2 *f, int nf, double *out);
void mg_coarse_solve_impl(dwf_ctx *c, int level, void *x, const void *b);
void mg_coarse_solve_static_impl(dwf_ctx *c, int level, void *x, const void *b);

// ---- transfer.cu ----
// c[Vc][nv] = R f  (R = P^+) ; f = P c (accumulate: f += P c)
template <typename R> void restrict_(dwf_ctx *c, const Level &L, C<R> *cout, const C<R> *fin, const C<R> *Q);
template <typename R> void prolong_(dwf_ctx *c, const Level &L, C<R> *fout, const C<R> *cin, const C<R> *Q, bool accumulate);
// the same with an FP16 copy of the basis (FP32 fields and arithmetic)
void restrict_h(dwf_ctx *c, const Level &L, float2 *cout, const float2 *fin, const __half2 *Q);
void prolong_h(dwf_ctx *c, const Level &L, float2 *fout, const float2 *cin, const __half2 *Q, bool accumulate);
void basis_to_half(dwf_ctx *c, __half2 *out, const float2 *in, int64_t n);
// batched transfers: nrhs fine fields <-> nrhs coarse fields, basis read once per 12 RHS
template <typename R> void restrict_batch(dwf_ctx *c, const Level &L, C<R> *cout, const C<R> *fin, const C<R> *Q, int nrhs);
template <typename R>
void prolong_batch(dwf_ctx *c, const Level &L, C<R> *fout, const C<R> *cin, const C<R> *Q, int nrhs, bool accumulate);
// G[Vc][nv][nv] = block inner products <A_k, B_l> over each block (FP64 accumulate)
template <typename R> void block_gram(dwf_ctx *c, const Level &L, double2 *G, const C<R> *A, const C<R> *B);
// In-place block orthonormalisation of the nv fields Q (CholQR2, FP64); returns false on breakdown
template <typename R> bool block_orthonormalise(dwf_ctx *c, Level &L, C<R> *Q);
// Q[2j] = (1 + Gamma)/2 v_j, Q[2j+1] = (1 - Gamma)/2 v_j  (Gamma = g5 R5 on the fine level,
// +-1 on even/odd components of a coarse level); split = false copies v_j to Q[j]
template <typename R> void gamma_split(dwf_ctx *c, const Level &L, C<R> *Q, const double2 *v, int nadapt, bool split);

// ---- coarse.cu ----
// y = A_l c on coarse level l (l >= 1), or A_l^+ c
template <typename R> void coarse_apply(dwf_ctx *c, const Level &L, C<R> *y, const C<R> *x, bool dag);
// Build the Galerkin coarse operator Y (FP64) of level Lc = l+1 from level L's
// basis Q (W: scratch of L.nv fields of level L, same precision)
template <typename R> void build_coarse_from(dwf_ctx *c, Level &L, Level &Lc, const C<R> *Q, C<R> *W);
// refresh the reduced-precision copies of Y on level l
void convert_coarse_links(dwf_ctx *c, Level &L);
// ---- coarse_sq.cu ---- the squared operator's coarse stencil (Sec. 4):
// Y of level Lc = 1 as [V][33][n][n] = P^+ D^+ D P from the fine basis Q
// (W: scratch of L.nv fine fields, same precision)
template <typename R> void build_squared_coarse(dwf_ctx *c, Level &L, Level &Lc, const C<R> *Q, C<R> *W);
// coarse offsets of the 33-point stencil: off[d][mu] in {-1, 0, 1}
void squared_offsets(int off[33][4]);

// ---- coarse_gcr.cu ----  fused coarsest-level GCR (one cooperative launch)
bool coarse_gcr_fused_ok(const Level &L, int restart);
// ---- coarse_gcr_sq.cu ---- the same kernel on the 33-point stencil
template <typename R>
void coarse_gcr_launch_squared(dwf_ctx *c, const Level &L, C<R> *x, const C<R> *b, C<R> *r, C<R> *Z, C<R> *W,
                               double2 *part, int *iters, double tol, int maxiter, int restart);
// ---- coarse_gcr_batch.cu ---- the same solve for nb <= 16 right-hand sides in lockstep
bool coarse_gcr_batch_ok(const Level &L, int restart, int nb);
size_t coarse_gcr_batch_part_bytes(dwf_ctx *c);
template <typename R>
void coarse_gcr_fused_batch(dwf_ctx *c, const Level &L, C<R> *x, const C<R> *b, int nb, C<R> *r, C<R> *Z, C<R> *W,
                            double2 *part, int *iters, double tol, int maxiter, int restart);
size_t coarse_gcr_part_bytes(dwf_ctx *c);
// ---- coarse_gcr_tc.cu ---- the batched solve with the BF16 stencil on the tensor cores
// (FP32 fields, 9-point stencil, Nvec in {8, 16, 24, 32}, nb <= 16, restart <= 16)
bool coarse_gcr_tc_ok(dwf_ctx *c, const Level &L, int restart, int nb);
void coarse_gcr_tc(dwf_ctx *c, const Level &L, float2 *x, const float2 *b, int nb, float2 *r, float2 *Z, float2 *W,
                   double2 *part, int *iters, double tol, int maxiter, int restart);
void build_tc_images(dwf_ctx *c, Level &L);
// throws DWF_ETIMEOUT when a tensor-core solve since the last check gave up a bounded wait
void check_tc_timeout(dwf_ctx *c);
template <typename R>
void coarse_gcr_fused(dwf_ctx *c, const Level &L, C<R> *x, const C<R> *b, C<R> *r, C<R> *Z, C<R> *W, double2 *part,
                      int *iters, double tol, int maxiter, int restart);

template <typename T> void norm2_b(dwf_ctx *c, BatchScratch &bs, int base, int stride, const T *x, int64_t n, int nrhs);
template <typename T>
void multidot_b(dwf_ctx *c, BatchScratch &bs, int base, int stride, T *const *V, int k, const T *w, int64_t n, int nrhs);
template <typename T> void multiaxpy_b(dwf_ctx *c, T *w, T *const *V, int k, int base, int stride, double sgn, int64_t n, int nrhs);
// r = rin - a w (rin may be r), a = |z|^2 / |w|^2 from the slots
template <typename T>
void cg_r_b(dwf_ctx *c, T *r, const T *rin, const T *w, int base, int stride, int izz, int iww, int64_t n, int nrhs);
// x += a pin (x = a pin with xinit); unless last, pout = z + beta pin (pin may be pout)
template <typename T>
void cg_px_b(dwf_ctx *c, T *x, T *pout, const T *pin, const T *z, int base, int stride, int izz, int iww, int inew,
             int64_t n, int nrhs, bool last, bool xinit);
// CGNR direction update with x += a p deferred: np (<= CG_MAXDEFER) pending
// directions pend[] with their steps in scalar slots ia, ia+1, ...; mode 0
// defers pin as well (its step into slot ia + np), mode 1 adds every pending
// step and a pin to x and updates the direction, mode 2 only adds them (last iteration)
constexpr int CG_MAXDEFER = 3;
template <typename T>
void cg_pxd_b(dwf_ctx *c, T *x, T *pout, const T *pin, T *const *pend, int np, const T *z, int base, int stride,
              int izz, int iww, int inew, int ia, int64_t n, int nrhs, int mode);
// x += the solution of k CGNR iterations expressed in their stored
// normal-equations residuals Z[0..k-1] (k <= 32); |z_j|^2 in slot zb + j and
// |w_j|^2 = |D p_j|^2 in slot wb + j of each right-hand side's block
template <typename T>
void cg_combine_b(dwf_ctx *c, T *x, T *const *Z, int k, int base, int stride, int zb, int wb, int64_t n, int nrhs);
// End of a chunk of m CGNR iterations from k0 that kept their residuals
// Z[t-1] = z_{k0+t} (t = 1 .. m-1, and m with next): x (+)= sum_t a_t p_t with
// p the chunk's first direction, and with next p <- the next chunk's first
// direction; norms in the slot rings zb + (k0 + t) % rs and wb + (k0 + t) % rs
template <typename T>
void cg_chunk_b(dwf_ctx *c, T *x, T *p, T *const *Z, int m, bool next, bool xinit, int base, int stride, int zb, int wb,
                int k0, int rs, int64_t n, int nrhs);
template <typename T> void gcr_wr_b(dwf_ctx *c, T *w, T *res, const double *sc, const double2 *al, int64_t n, int nrhs);
template <typename T> void combo_b(dwf_ctx *c, T *x, T *const *V, int k, const double2 *g, int64_t n, int nrhs);

// ---- blas2.cu ----  (host scalars; FP64 accumulate inside reductions)
template <typename T> void caxpy(dwf_ctx *c, T *y, double2 a, const T *x, int64_t n);       // y += a x
template <typename T> void cxpay(dwf_ctx *c, T *y, double2 a, const T *x, int64_t n);       // y = x + a y
template <typename T> void rscale(dwf_ctx *c, T *x, double a, int64_t n);                   // x *= a
// y_out(T) += a * x(U) with precision conversion (x may be another precision)
template <typename T, typename U> void caxpy_mixed(dwf_ctx *c, T *y, double2 a, const U *x, int64_t n);
// w += sum_i beta_i V_i, k <= 32 (pointers and coefficients from the host)
template <typename T> void multiaxpy(dwf_ctx *c, T *w, const double2 *beta, T *const *V, int k, int64_t n);
constexpr int MAX_RESTART = 64;
// device-coefficient solver updates (scalar slots index ctx->scal)
template <typename T> void cg_xr(dwf_ctx *c, T *x, T *r, const T *p, const T *w, int izz, int iww, int64_t n);
template <typename T> void cg_p(dwf_ctx *c, T *p, const T *z, int inew, int iold, int64_t n);
template <typename T> void multiaxpy_dev(dwf_ctx *c, T *w, T *const *V, int k, int ibase, double sgn, int64_t n);
template <typename T> void gcr_step(dwf_ctx *c, T *x, T *r, T *z, T *w, int iww, int ia, int64_t n);
// x = a * x + b * y (real a, complex b) fused for two pairs: used by GCR updates
template <typename T> void gauss_fill(dwf_ctx *c, double2 *out, int nfields, int64_t nelem, int Ls, int64_t V,
                                      bool canonical_fine, uint32_t seed, uint32_t stream);

// ---- net.cu ---- learned near-null proposal (include/dwfnet.h)
dwf_net *net_create_impl(dwf_ctx *c, const dwf_net_shape &s);
void net_set_params_impl(dwf_net *net, const void *p, bool dev);
void net_get_params_impl(dwf_net *net, void *p, bool dev);
void net_forward_impl(dwf_net *net, dwf_ctx *c, const void *input, bool input_dev, unsigned seed, double2 *out);
double net_loss_grad_impl(dwf_net *net, dwf_ctx *c, const void *input, bool input_dev, unsigned seed,
                          const double2 *targets, int nt, const int block[4], void *grad, bool grad_dev);
void net_adam_impl(dwf_net *net, double lr, double b1, double b2, double eps);
void net_refine_impl(dwf_net *net, dwf_ctx *c, const double2 *fields, int B, double2 *out);
double net_refine_loss_grad_impl(dwf_net *net, dwf_ctx *c, const double2 *fields, int B, const double2 *targets, int nt,
                                 const int block[4], void *grad, bool grad_dev);
bool net_is_refiner(const dwf_net *net);
long long net_nparams(const dwf_net *net);
void net_set_wprec_impl(dwf_net *net, dwf_prec prec);
int net_nout(const dwf_net *net);
void net_free(dwf_net *net);

}  // namespace dwf
