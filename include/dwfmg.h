/*
 * dwfmg — adaptive multigrid for the 5D Shamir domain-wall fermion operator
 * on one NVIDIA GB300 GPU (sm_103a).
 *
 * The method is that of Cohen, Brower, Clark, Osborn, "Multigrid Algorithms
 * for Domain-Wall Fermions" (Lattice 2011): solve D x = b (Sec. 1: the
 * problem A x = b with residual r = A x - b) with flexible GCR (Sec. 3)
 * preconditioned by a V-cycle (Sec. 2: pre-smooth, restrict, coarse solve,
 * prolong, post-smooth) whose coarse spaces are spanned by adaptively found
 * near-null vectors cut into blocks that cover the whole fifth dimension
 * (Sec. 2).
 *
 * Conventions used throughout
 * ---------------------------
 * Lattice: dims[4] = {X, Y, Z, T}; 4D site index site = ((t*Z + z)*Y + y)*X + x.
 * Operator (Sec. 2 names the Shamir domain-wall operator; Sec. 4 its 11-site
 * one-hop stencil; the explicit form below is the standard unnormalised
 * Shamir operator):
 *   (D psi)(x,s) = (5 - M5) psi(x,s)
 *       - 1/2 sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu,s) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu,s) ]
 *       - P_- psi(x,s+1) - P_+ psi(x,s-1),
 *   where at s = Ls-1 the term -P_- psi(x,Ls) becomes +mf P_- psi(x,0) and at
 *   s = 0 the term -P_+ psi(x,-1) becomes +mf P_+ psi(x,Ls-1).  Gamma matrices
 *   in the chiral (DeGrand-Rossi) basis, g_5 = diag(1,1,-1,-1), P_+- = (1 +- g_5)/2.
 *   Links are periodic; the fermion is periodic in x, y, z and, if
 *   antiperiodic_t != 0, antiperiodic in t.
 * Links (input): complex128, U[site][mu][a][b] (row a, column b), mu = 0..3
 *   for x, y, z, t.  They must be SU(3) (unitary, det 1): the FP32 copy keeps
 *   two rows and rebuilds the third.
 * Canonical fermion layout (dwf_pack / dwf_unpack): complex, index
 *   ((s*V + site)*4 + spin)*3 + colour, s slowest.
 * Internal fermion layout (every other call): complex, index
 *   (site*12 + spin*3 + colour)*Ls + s, s fastest.  FP64 = interleaved
 *   double pairs, FP32 = interleaved float pairs.  With nrhs > 1 the nrhs
 *   fields follow one another in memory.
 *
 * Memory and ownership: every pointer argument named *_dev must be device
 * memory of the current CUDA device; arguments documented as "host or
 * device" are inspected with cudaPointerGetAttributes and staged through
 * library-owned device buffers when they are host memory.  The caller owns
 * all buffers it passes in; the library never frees them.  The context owns
 * everything it allocates (link copies, near-null vectors, coarse operators,
 * workspaces) and frees it in dwf_destroy.
 *
 * Streams: all work of a context runs on the stream given to dwf_create.
 * dwf_apply, dwf_pack and dwf_unpack are asynchronous; mg_setup and mg_solve
 * synchronise the stream before they return their status.
 *
 * Errors: calls return a dwf_status and never throw.  After DWF_ECUDA the
 * context is left in an error state and every later call returns DWF_ESTATE.
 * There is no CPU fallback: without a CUDA device dwf_create fails.
 */
#ifndef DWFMG_H
#define DWFMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dwf_ctx dwf_ctx;

typedef enum {
    DWF_OK = 0,
    DWF_EINVAL = -1,      /* bad argument (sizes, null pointers, unsupported combination) */
    DWF_ECUDA = -2,       /* a CUDA call failed; the context is unusable */
    DWF_ENOMEM = -3,      /* device allocation failed */
    DWF_ENOCONV = -4,     /* solver hit its iteration limit; x holds the best iterate */
    DWF_EBREAKDOWN = -5,  /* Krylov or Gram-Schmidt breakdown (zero or dependent vectors) */
    DWF_ENAN = -6,        /* NaN or Inf met in a norm */
    DWF_ETIMEOUT = -7,    /* a bounded device-side wait gave up */
    DWF_ESTATE = -8       /* wrong call order, or context in error state */
} dwf_status;

typedef enum { DWF_F64 = 0, DWF_F32 = 1, DWF_BF16 = 2, DWF_F16 = 3 } dwf_prec;

/* Multigrid parameters.  The paper leaves the smoothers S1, S3, the coarse
 * solver S2 and the iteration counts open (Sec. 2); mg_default_params fills
 * in this library's choices.  Level 0 is the fine lattice. */
typedef struct {
    int nu_pre;             /* nu_1: CGNR smoothing steps before restriction (default 0) */
    int nu_post;            /* nu_3: CGNR smoothing steps after prolongation (default 8) */
    double coarse_tol;      /* S2 relative tolerance on intermediate levels (0.1) */
    int coarse_maxiter;     /* (24) */
    double coarsest_tol;    /* S2 relative tolerance on the coarsest level (0.1) */
    int coarsest_maxiter;   /* (64) */
    int coarse_restart;     /* GCR restart length of S2 (16) */
    int outer_restart;      /* outer flexible GCR restart length, <= 64 (20) */
    int outer_maxiter;      /* (500) */
    int setup_iters0;       /* CGNR iterations on D x = 0 for the initial vectors, at most (1000) */
    double setup_tol0;      /* ... or until |D x| <= setup_tol0 |D x_0|, tested every 8 iterations (1e-6) */
    int setup_sweeps;       /* inverse-iteration sweeps with the current multigrid (0) */
    int setup_sweep_iters;  /* MG-GCR iterations per vector and sweep, at most (8) */
    double setup_sweep_tol; /* MG-GCR relative tolerance of a sweep's solve D x = v (0.1) */
    int split;              /* 1: each vector split into Gamma = +-1 halves, Nvec/2 vectors (1) */
    dwf_prec smoother_prec; /* F64 (plain method) or F32 (mixed) for the fine V-cycle (F64) */
    dwf_prec coarse_prec[4];/* link precision of each coarse level's stencil: F64, F32, BF16, F16 */
    dwf_prec basis_prec;    /* with smoother_prec = F32: F16 keeps an FP16 copy of the block basis for
                               the V-cycle's restriction and prolongation (FP32 arithmetic), F32 none (F32) */
    uint32_t seed;          /* Philox seed of the random start vectors when none are given */
    int cycle;              /* S2 on intermediate levels (3+ levels): 0 = GCR preconditioned by the next
                               V-cycle (a K-cycle), 1 = two V-cycles, x = V(b), x += V(b - A x): the
                               W-cycle of Sec. 2 (0) */
    int coarsen;            /* coarse operator: 0 = R D P, the 9-point stencil of the unsquared
                               operator; 1 = P^+ D^+ D P, the coarsened squared operator that
                               Sec. 4 uses (33-point stencil: offset 0, the 8 one-hop offsets and
                               the 24 two-hop diagonals; two levels only, every block extent >= 2
                               except along lattice directions of extent 1;
                               the V-cycle restricts D^+ r instead of r, and several right-hand
                               sides are solved one after another) (0) */
    int graph;              /* 1: the batched V-cycle (FP32, two levels, several right-hand sides)
                               is captured once per solve call, batch width and direction slot as a
                               CUDA graph and replayed; 0: launched kernel by kernel.  Ignored for a
                               lattice of a batch context (dwf_create with nlat > 1) (1) */
} mg_params;

typedef struct {
    int iters;                  /* outer GCR iterations */
    int restarts;               /* outer cycles (each ends with an FP64 true residual) */
    long long fine_applies_f64; /* fine D applications in FP64 (incl. D^+ in CGNR) */
    long long fine_applies_f32; /* fine D applications in FP32 */
    long long coarse_applies[4];/* coarse operator applications per level 1..3 */
    double true_res;            /* |b - D x| / |b| in FP64 at return */
    double seconds;             /* wall time of the call */
} mg_stats;

/* Fill p with the defaults listed above. */
void mg_default_params(mg_params *p);

/* Create a context for nlat independent lattices of the same Ls, M5 and mf
 * (Sec. 1-2 state the problem D x = b for one lattice; a batch holds several
 * such problems, e.g. lattices of uneven size, behind one handle).
 *   nlat        number of lattices (1 <= nlat <= 64)
 *   dims        nlat rows of X, Y, Z, T (each >= 1)
 *   Ls          fifth-dimension extent (1 <= Ls <= 128)
 *   M5, mf      domain-wall height and quark mass
 *   links       nlat pointers, each complex128 U[V_i][4][3][3] of lattice i,
 *               host or device; copied
 *   antiperiodic_t  nonzero: antiperiodic fermion boundary in t
 *   stream      cudaStream_t to run on (NULL = legacy default stream)
 * With nlat > 1 every field argument of dwf_apply, dwf_pack, dwf_unpack,
 * mg_setup (start) and mg_solve holds the lattices one after another: the
 * nrhs fields of lattice 0, then those of lattice 1, ...  Each lattice runs
 * on a stream the library creates (joined to `stream` before the call
 * returns for the asynchronous calls); mg_setup and mg_solve drive the
 * lattices concurrently from host threads, with the same parameters for
 * every lattice (each block must divide every lattice).  Every other call
 * takes one lattice: get its handle with dwf_lattice.
 * Returns DWF_EINVAL for bad sizes, DWF_ENOMEM / DWF_ECUDA on CUDA failure. */
dwf_status dwf_create(dwf_ctx **out, int nlat, const int (*dims)[4], int Ls, double M5, double mf,
                      const void *const *links, int antiperiodic_t, void *stream);

/* The context of lattice i of a batch (for nlat = 1, i = 0 gives ctx itself).
 * The handle is borrowed: it stays valid until dwf_destroy(ctx) and must not
 * be destroyed by the caller.  Its calls run on the lattice's own stream. */
dwf_status dwf_lattice(dwf_ctx *ctx, int i, dwf_ctx **out);

/* out = D in (dagger = 0) or D^+ in (dagger != 0) for nrhs fields in the
 * internal layout, in FP64 or FP32 (prec = DWF_F64 or DWF_F32).  Fine
 * operator of Sec. 2 / Sec. 4 (the 11-site stencil).  out and in are
 * device pointers and must not overlap.  Asynchronous.  On a batch: nrhs
 * fields of every lattice, lattices one after another. */
dwf_status dwf_apply(dwf_ctx *ctx, void *out_dev, const void *in_dev, dwf_prec prec, int dagger,
                     int nrhs);

/* Convert nrhs fields between the canonical layout (complex128, s slowest)
 * and the internal layout in precision prec.  Both pointers device memory. */
dwf_status dwf_pack(dwf_ctx *ctx, void *internal_dev, const void *canonical_dev, dwf_prec prec,
                    int nrhs);
dwf_status dwf_unpack(dwf_ctx *ctx, void *canonical_dev, const void *internal_dev, dwf_prec prec,
                      int nrhs);

/* Adaptive multigrid setup (Sec. 2).
 *   levels      total number of levels including the fine one (2 or 3)
 *   nvec        coarse components per site for each coarse level (levels-1
 *               entries); with split = 1 each must be even and Nvec/2 adaptive
 *               vectors are used
 *   block       4D block (bx, by, bz, bt) of each transfer (levels-1 entries);
 *               each must divide the lattice of its level.  Blocks always
 *               cover the whole fifth dimension (Sec. 2).
 *   opt         parameters, NULL = mg_default_params
 *   start       optional random start vectors of the fine level: Nvec/2 (split)
 *               or Nvec fields in the canonical layout, complex128, host or
 *               device.  NULL: drawn on the device from Philox-4x32-10 with
 *               opt->seed.
 * Synchronous.  DWF_EBREAKDOWN if block Gram-Schmidt meets dependent
 * vectors.  On a batch: every lattice gets the same levels, nvec, block
 * and parameters; start (if given) holds each lattice's vectors in turn. */
dwf_status mg_setup(dwf_ctx *ctx, int levels, const int *nvec, const int (*block)[4],
                    const mg_params *opt, const void *start);

/* Solve D x = b to |b - D x| / |b| <= tol (true residual, FP64) with
 * flexible GCR preconditioned by one V-cycle per iteration (Sec. 2, Sec. 3).
 *   b, x        nrhs fields in the internal layout, complex128, host or
 *               device; x holds the initial guess on entry and the solution
 *               on return (also on DWF_ENOCONV: the best iterate).
 *   stats       optional, filled on return (totals over the nrhs solves).
 * Synchronous.  On a batch: nrhs right-hand sides per lattice, lattices one
 * after another in b and x; stats sums iterations and applications over
 * the lattices and gives the largest true residual; the status is the
 * first lattice's that is not DWF_OK. */
dwf_status mg_solve(dwf_ctx *ctx, const void *b, void *x, double tol, int nrhs, mg_stats *stats);

/* ---- Component calls --------------------------------------------------
 * Each runs one step of the V-cycle on its own, for parity checks against a
 * reference and for diagnostics.  They need a completed mg_setup.  Levels
 * count from 0 (the fine lattice).  A coarse field of level l >= 1 is
 * [site][Nvec] complex over that level's lattice (site index x fastest).
 * All fields are device memory; FP64 unless stated.  Asynchronous unless
 * stated. */

/* Lattice extents and components per site of level l (fine: 12 per s). */
dwf_status mg_level_info(dwf_ctx *ctx, int level, int dims_out[4], int *ncomp_out);

/* Copy the Nvec block-orthonormal basis fields q_k of level l (Sec. 1:
 * columns of the prolongator P, R = P^+, R P = 1_c), FP64. */
dwf_status mg_get_vectors(dwf_ctx *ctx, int level, void *out_dev);

/* Copy the coarse stencil of level l >= 1: Y[site][d][k][m], d = 0 self,
 * 1+2mu (+mu), 2+2mu (-mu), FP64 (Sec. 2: the coarse operator R A P).  With
 * coarsen = 1 the stencil has 33 points: d as above for d < 9, then
 * d = 9 + 4 p + 2 a + b for the diagonal +-mu +-nu, p the rank of (mu, nu) in
 * (0,1), (0,2), (0,3), (1,2), (1,3), (2,3), a = 1 for -mu, b = 1 for -nu
 * (out holds V * 33 * n * n complex numbers). */
dwf_status mg_get_coarse_links(dwf_ctx *ctx, int level, void *out_dev);

/* coarse_out (level l+1) = R fine_in (level l);  fine_out = P coarse_in. */
dwf_status mg_restrict(dwf_ctx *ctx, int level, void *coarse_out_dev, const void *fine_in_dev);
dwf_status mg_prolong(dwf_ctx *ctx, int level, void *fine_out_dev, const void *coarse_in_dev);

/* out = A_l in (or A_l^+ in) with the coarse stencil of level l >= 1 in the
 * level's link precision; prec = DWF_F64 or DWF_F32 for the fields.  The
 * squared operator's stencil (coarsen = 1) is Hermitian: dagger is ignored. */
dwf_status mg_coarse_apply(dwf_ctx *ctx, int level, void *out_dev, const void *in_dev, int dagger, dwf_prec prec);

/* x = S2(R A P, b) on the coarsest level (Sec. 2, third step of the
 * V-cycle): restarted GCR on the coarse stencil from x = 0 to the relative
 * tolerance coarsest_tol (at most coarsest_maxiter iterations), as one
 * cooperative kernel.  x and b are coarse fields of that level in the
 * V-cycle precision (FP64 for smoother_prec = F64, FP32 for F32).
 * Synchronous. */
dwf_status mg_coarse_solve(dwf_ctx *ctx, int level, void *x_dev, const void *b_dev);

/* Same result as mg_coarse_solve, for callers that cannot allocate device
 * memory when they solve (a host framework that gives the library a fixed
 * device-memory budget, or a runtime whose allocator must not be re-entered
 * from inside the solve).  The paper has no counterpart: this is
 * an interface choice of this library.  It allocates nothing: all scratch of
 * the solver lives in one static device array of 8 MiB that every GPU
 * loading the library holds until the process exits.
 *   Limits: coarse_restart <= 16, and
 *     256 + roundup256(1632 * SM count) + (1 + 2*coarse_restart) * vector bytes
 *   must not exceed 8 MiB, a vector being one coarse field in the V-cycle
 *   precision (e.g. 512 sites x 24 components in FP32 at restart 16:
 *   33 x 98,304 B = 3.1 MiB, plus 0.24 MiB of FP64 partial sums on 152
 *   SMs); larger requests return DWF_EINVAL.
 *   Set-up: the first call on a device looks up the array's device address
 *   (the context's device must be current); make that first call before
 *   any stream capture.
 *   Sharing: every call uses the same array (the iteration counter is
 *   cleared at each call); calls that overlap on the GPU -- on different
 *   streams or contexts of the same device -- race and must be serialised
 *   by the caller.
 * x and b are device fields as for mg_coarse_solve and must not overlap
 * (DWF_EINVAL).  Synchronous. */
dwf_status mg_coarse_solve_static(dwf_ctx *ctx, int level, void *x_dev, const void *b_dev);

/* x = one fine-level V-cycle applied to b (Sec. 2), run in the smoother
 * precision; x and b are FP64.  Synchronous. */
dwf_status mg_vcycle(dwf_ctx *ctx, void *x_dev, const void *b_dev);

/* The adaptive vectors a finished setup built level `level` from (Nvec/2
 * with split, else Nvec fields of that level), globally orthonormal, before
 * the Gamma split and block orthonormalisation: complex128, internal
 * layout, device.  Synchronous. */
dwf_status mg_get_adaptive_vectors(dwf_ctx *ctx, int level, void *out_dev);

/* ---- Low-mode diagnostic (Sec. 2, Fig. 1: the overlap of the low modes
 * with the coarse space) -------------------------------------------------
 * dwf_lowest_modes: the k (1..32) smallest eigenpairs of D^+ D by subspace
 * iteration on (D^+ D)^-1 = D^-1 Gamma D^-1 Gamma, each D^-1 a multigrid
 * solve of the current setup (mg_setup must have completed), with
 * Rayleigh-Ritz on the iterated subspace; start vectors from Philox with key
 * (seed, 8).  Stops when every relative residual |A v - lambda v| / lambda
 * is <= tol or after max_iters iterations.  evals: k doubles (host,
 * ascending); evecs_dev: k complex128 fine fields, internal layout, device,
 * orthonormal; resid: NULL or k doubles (host); iters: NULL or the count.
 * mg_coarse_overlap: for nfields complex128 fields of level `level`
 * (internal layout, device) the shares |P^+ v|^2 / |v|^2 of each inside the
 * coarse space of that level's transfer (host doubles).  Both synchronous. */
dwf_status dwf_lowest_modes(dwf_ctx *ctx, int k, int max_iters, double tol, unsigned int seed, double *evals,
                            void *evecs_dev, double *resid, int *iters);
dwf_status mg_coarse_overlap(dwf_ctx *ctx, int level, const void *fields_dev, int nfields, double *overlap);

/* The V-cycle of mg_vcycle (Sec. 2) for nrhs right-hand sides stored one
 * after another (nrhs fine FP64 fields each for x and b).  With an FP32
 * V-cycle on two levels and nu_1 = 0 the right-hand sides go through the
 * fine level together (one Dslash launch, one read of the transfer basis
 * per 12 of them) and their coarsest solves run concurrently; otherwise
 * they run one after another.  Each x_r equals what mg_vcycle gives for
 * b_r up to rounding order.  x and b must not overlap.  Synchronous. */
dwf_status mg_vcycle_batch(dwf_ctx *ctx, void *x_dev, const void *b_dev, int nrhs);

/* ---- Measurement -------------------------------------------------------
 * An optional profiler brackets every launch of the timed kernel classes
 * with CUDA events on the context's stream.  dwf_profile(ctx, 1) clears the
 * records and starts recording, dwf_profile(ctx, 0) stops; dwf_profile_read
 * synchronises the stream and returns the number of launches and their
 * summed device time for one class.  Classes: 0 = fine D in FP64, 1 = fine
 * D in FP32, 2 = restriction, 3 = prolongation, 4 = coarse stencil, 5 = fine
 * D in FP32 that combines its result with a second field (the V-cycle's
 * residual b - D x, the smoother's z - a D^+ w). */
dwf_status dwf_profile(dwf_ctx *ctx, int enable);
dwf_status dwf_profile_read(dwf_ctx *ctx, int kernel_class, long long *launches, double *total_ms);
/* The number of fields (right-hand sides) the recorded launches of one class
 * processed: a batched launch over nrhs fields counts nrhs (classes 0, 1, 5:
 * fine D applications; 2, 3: batched transfers count their right-hand sides). */
dwf_status dwf_profile_units(dwf_ctx *ctx, int kernel_class, long long *units);

/* Number of kernels this library has launched in the process so far. */
unsigned long long dwf_launch_count(void);

/* Description of the last error raised on this thread (diagnostics). */
const char *dwf_last_error(void);

/* The paper's comparison solver (Sec. 3: conjugate gradient on the squared
 * operator): CG on D^+ D x = D^+ b in precision prec (DWF_F64 or DWF_F32),
 * with a reliable update (FP64 true residual, search direction kept) every
 * 200 iterations, until
 * |b - D x| / |b| <= tol or maxiter iterations.  Same buffers and stats as
 * mg_solve (iters = CG iterations; each costs one D and one D^+).  Needs no
 * mg_setup.  Synchronous. */
dwf_status dwf_cg_solve(dwf_ctx *ctx, const void *b, void *x, double tol, int maxiter, int nrhs, dwf_prec prec,
                        mg_stats *stats);

/* Description of a status code (static string). */
const char *dwf_strerror(dwf_status s);

/* Release everything the context owns (for a batch, every lattice's
 * context and stream).  Safe on NULL. */
void dwf_destroy(dwf_ctx *ctx);

/* ---- Environment switches ----------------------------------------------
 * Unset, every switch selects the production path.  They exist for
 * measurements and tests; each is read once per process except where noted.
 *   DWF_DSLASH_PAIR=0        FP32 Dslash with one fifth-dimension slice per
 *                            thread instead of the paired kernel (which also
 *                            disables the fused norm and residual epilogues)
 *   DWF_DSLASH_PAIR_MINB=4   paired FP32 Dslash in 128-thread CTAs, 4 per SM
 *                            (default: 64 threads, 8 per SM)
 *   DWF_DSLASH_MINB=6        one-slice Dslash at 80 registers, 6 CTAs per SM
 *   DWF_BATCH=0              several right-hand sides solved one at a time
 *   DWF_COARSE_BATCH=0       the batched V-cycle's coarsest solves one
 *                            right-hand side per cooperative launch
 *   DWF_SMOOTHER_HISTORY=0   the batched CGNR with a direction vector instead
 *                            of the form that keeps its residuals (read at
 *                            every solve call)
 *   DWF_TC_FORCE_WAIT=n      test hook: the first n launches of the
 *                            tensor-core coarsest solver begin with a wait
 *                            that runs out after about one second (the call
 *                            returns DWF_ETIMEOUT)
 *   DWF_VERBOSE=1            the coarsest solver's grid tuning is printed
 */

#ifdef __cplusplus
}
#endif

#endif /* DWFMG_H */
