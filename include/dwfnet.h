/* dwfnet: learned near-null proposal for the adaptive multigrid setup of
 * dwfmg (GB300, sm_103a).
 *
 * The paper finds the near-null vectors of its adaptive setup (Sec. 2) by
 * relaxing on D x = 0 from random vectors.  This interface adds a small
 * gauge-covariant convolutional network that proposes those vectors from the
 * links; the setup then refines the proposal with a few relaxation
 * iterations (mg_setup with the proposal as its start vectors).  The paper
 * has no network: the design below is this library's.
 *
 * Network (complex FP32 arithmetic on the GPU):
 *   input   h_0: c_in channels x 4 spins x 3 colours per 4D site, Gaussian
 *           from Philox-4x32-10 (or given by the caller)
 *   layer   a_{l+1}(x) = sum_{d=0..8} W_l[d] (T_d h_l)(x), with the parallel
 *           transports T_0 h(x) = h(x), T_{+mu} h(x) = U_mu(x) h(x+mu),
 *           T_{-mu} h(x) = U_mu(x-mu)^+ h(x-mu) (periodic, no fermion
 *           boundary sign); W_l[d] acts on (channel, spin), never on colour
 *   gate    h_{l+1} = a_{l+1} t/(1+t), t = sum over colour of |a_{l+1}|^2
 *           for each (channel, spin, site)
 *   head    v_j(x, s, spin, colour) = sum_{c, spin'} Hd[j][s][spin][c][spin']
 *           h_L(x, c, spin', colour),  j < nout, s < Ls
 * so the outputs transform like fermion fields under gauge transformations.
 *
 * Parameters: one complex128 vector, the concatenation in C order of
 *   W_0 [hidden][4][9][c_in][4], W_l [hidden][4][9][hidden][4] (l = 1 ..
 *   layers-1), Hd [nout][Ls][4][hidden][4];
 * direction d: 0 the site itself, 1 + 2 mu the +mu transport, 2 + 2 mu the
 * -mu transport (mu = 0..3 for x, y, z, t).
 *
 * Loss (training against the adaptive setup's vectors): the outputs are
 * split by Gamma = gamma_5 R_5 into (1 +- Gamma)/2 v_j (as mg_setup splits
 * its vectors) and cut into the 4D blocks of the transfer (blocks cover all
 * of Ls).  For target fields q_c and every block b,
 *   L_b = min_Y || Q_b - H_b Y ||_F^2,
 * and L = sum_b L_b / (number of blocks * number of targets).  Gradients are
 * dL/d(conj theta) for the complex parameters theta.
 *
 * Layouts: fine fields as in dwfmg.h (canonical or internal as stated); the
 * input h_0 is complex128 [c_in][4][V][3] with the 4D site index of dwfmg.h.
 * Every call runs on the stream of the context it is given and synchronises
 * before returning.  Errors as in dwfmg.h.
 */
#ifndef DWFNET_H
#define DWFNET_H

#include "dwfmg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dwf_net dwf_net;

typedef struct {
    int c_in;    /* input channels (>= 1) */
    int hidden;  /* hidden channels (>= 1) */
    int layers;  /* convolution layers (>= 1); the first maps c_in -> hidden */
    int nout;    /* output fine fields: Nvec/2 of the setup it serves */
    int Ls;      /* fifth extent of the lattices it is applied to */
} dwf_net_shape;

/* A network on the device of ctx, parameters zero.  The network may then be
 * used with any context of that device whose Ls equals shape->Ls. */
dwf_status net_create(dwf_ctx *ctx, const dwf_net_shape *shape, dwf_net **out);

/* Number of complex parameters. */
dwf_status net_num_params(const dwf_net *net, long long *count);

/* Copy the parameters in or out: complex128, host or device. */
dwf_status net_set_params(dwf_net *net, const void *params);
dwf_status net_get_params(dwf_net *net, void *params);

/* out = the nout output fields for the links of ctx, complex128 canonical
 * layout (dwfmg.h), device memory: exactly what mg_setup takes as start
 * vectors.  input: h_0 (host or device) or NULL for Philox-4x32-10 with
 * key (seed, 7) drawn over the flat index of h_0. */
dwf_status net_forward(dwf_net *net, dwf_ctx *ctx, const void *input, unsigned int seed, void *out_dev);

/* The projection loss of the outputs against nt target fields (complex128,
 * internal layout, device: e.g. mg_get_vectors of a finished setup) on
 * blocks block[4] = (bx, by, bz, bt), and its gradient.  grad: NULL or the
 * parameter gradient (complex128, host or device).  The gradient is also kept
 * for net_adam.  DWF_EBREAKDOWN if the split outputs are linearly dependent
 * on a block. */
dwf_status net_loss_grad(dwf_net *net, dwf_ctx *ctx, const void *input, unsigned int seed,
                         const void *targets_dev, int nt, const int block[4], double *loss, void *grad);

/* Weight precision of the inference passes (net_forward, net_refine and the
 * learned setup): DWF_F32 (default) or DWF_BF16, weights rounded to BF16
 * (round to nearest even) with FP32 arithmetic and accumulation.  Training
 * (net_loss_grad, net_refine_loss_grad, net_adam) always uses the FP32 master
 * weights.  DWF_EINVAL for other precisions. */
dwf_status net_set_weight_precision(dwf_net *net, dwf_prec prec);

/* One Adam step (Kingma and Ba, 2015) on the real and imaginary parts of the
 * parameters with the gradient of the last net_loss_grad (the real gradient
 * of a complex parameter is 2 (Re G, Im G)). */
dwf_status net_adam(dwf_net *net, double lr, double beta1, double beta2, double eps);

void net_destroy(dwf_net *net);

/* Refinement mode: a network with c_in = Ls and nout = 1 improves given
 * fields instead of drawing them.  Field v_b enters with its fifth dimension
 * as the c_in channels, scaled by alpha = sqrt(Ls V 12)
 * (h_0[s][spin](x, colour) = alpha v_b(x, s, spin, colour), entries of order
 * one for a unit-norm field) and leaves as v_b + head(h_L) / alpha (a skip
 * connection: zero head weights return the input).  in_dev: nfields complex128 fine fields, internal layout, device
 * (e.g. mg_get_adaptive_vectors after a short setup); out_dev: nfields
 * complex128 fields, canonical layout, device. */
dwf_status net_refine(dwf_net *net, dwf_ctx *ctx, const void *in_dev, int nfields, void *out_dev);

/* The projection loss of net_refine's outputs (as net_loss_grad). */
dwf_status net_refine_loss_grad(dwf_net *net, dwf_ctx *ctx, const void *in_dev, int nfields, const void *targets_dev,
                                int nt, const int block[4], double *loss, void *grad);

/* The learned setup: mg_setup (dwfmg.h) started from the network's vectors,
 * which opt->setup_iters0 relaxation iterations then refine.  A proposal
 * network (nout = nvec[0]/2 with opt->split = 1, else nvec[0]) draws them
 * (net_forward with input NULL and this seed); a refinement network
 * (net_refine) improves the vectors of a first setup that relaxes random
 * vectors for pre_iters0 iterations.
 * Fallback to the plain adaptive setup: when probe_max_iters > 0, a probe
 * solve (a Gaussian source from Philox-4x32-10 with key (seed, 3), x = 0)
 * runs to the relative residual probe_tol; if it needs more than
 * probe_max_iters outer iterations or fails, the setup is redone from random
 * vectors with setup_iters0 = fallback_iters0, and *used_fallback (if not
 * NULL) is set to 1 (else 0).  Synchronous. */
dwf_status mg_setup_learned(dwf_ctx *ctx, dwf_net *net, unsigned int seed, int levels, const int *nvec,
                            const int (*block)[4], const mg_params *opt, int pre_iters0, int fallback_iters0,
                            double probe_tol, int probe_max_iters, int *used_fallback);

#ifdef __cplusplus
}
#endif

#endif
