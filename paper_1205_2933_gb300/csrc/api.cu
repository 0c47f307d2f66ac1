// C-ABI entry points of dwfmg (see include/dwfmg.h for the contract).
#include <cstring>
#include <exception>

#include "batch.cuh"
#include "dwf_internal.cuh"
#include "mg.cuh"

using dwf::Error;

namespace {

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

dwf_status fail(dwf_ctx *c, const Error &e) {
    if (c && (e.st == DWF_ECUDA)) c->sticky = DWF_ESTATE;
    if (c) dwf::set_last_error(e.msg);
    return e.st;
}

template <typename F> dwf_status guarded(dwf_ctx *c, F &&f) {
    if (c && !c->members.empty()) {
        dwf::set_last_error("a batch of lattices: this call takes one lattice (dwf_lattice)");
        return DWF_EINVAL;
    }
    if (c && c->sticky != DWF_OK) return DWF_ESTATE;
    try {
        return f();
    } catch (const Error &e) {
        return fail(c, e);
    } catch (const std::bad_alloc &) {
        return DWF_ENOMEM;
    } catch (...) {
        return DWF_ECUDA;
    }
}

}  // namespace

extern "C" {

void mg_default_params(mg_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nu_pre = 0;
    p->nu_post = 8;
    p->coarse_tol = 0.1;
    p->coarse_maxiter = 24;
    p->coarsest_tol = 0.1;
    p->coarsest_maxiter = 64;
    p->coarse_restart = 16;
    p->outer_restart = 20;
    p->outer_maxiter = 500;
    p->setup_iters0 = 1000;
    p->setup_tol0 = 1e-6;
    p->setup_sweeps = 0;
    p->setup_sweep_iters = 8;
    p->setup_sweep_tol = 0.1;
    p->split = 1;
    p->smoother_prec = DWF_F64;
    for (int i = 0; i < 4; ++i) p->coarse_prec[i] = DWF_F64;
    p->basis_prec = DWF_F32;
    p->seed = 1u;
    p->cycle = 0;
    p->graph = 1;
}

const char *dwf_strerror(dwf_status s) {
    switch (s) {
        case DWF_OK: return "success";
        case DWF_EINVAL: return "invalid argument";
        case DWF_ECUDA: return "CUDA error";
        case DWF_ENOMEM: return "out of device memory";
        case DWF_ENOCONV: return "solver did not converge within its iteration limit";
        case DWF_EBREAKDOWN: return "Krylov or Gram-Schmidt breakdown";
        case DWF_ENAN: return "NaN or Inf encountered";
        case DWF_ETIMEOUT: return "device-side wait timed out";
        case DWF_ESTATE: return "invalid call order or context in error state";
    }
    return "unknown status";
}

}  // extern "C"

namespace dwf {

dwf_status create_one(dwf_ctx **out, const int dims[4], int Ls, double M5, double mf, const void *links,
                      int antiperiodic_t, void *stream) {
    if (!out || !dims || !links) return DWF_EINVAL;
    *out = nullptr;
    for (int i = 0; i < 4; ++i)
        if (dims[i] < 1) return DWF_EINVAL;
    if (Ls < 1 || Ls > 128) return DWF_EINVAL;
    dwf_ctx *c = new dwf_ctx();
    dwf_status st = guarded(nullptr, [&]() -> dwf_status {
        int ndev = 0;
        DWF_CUDA(cudaGetDeviceCount(&ndev));
        DWF_REQUIRE(ndev > 0, DWF_ECUDA, "no CUDA device");
        DWF_CUDA(cudaGetDevice(&c->device));
        DWF_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
        for (int i = 0; i < 4; ++i) c->g.L[i] = dims[i];
        c->g.Ls = Ls;
        c->g.V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
        c->g.ap = antiperiodic_t ? 1 : 0;
        c->M5 = M5;
        c->mf = mf;
        c->stream = (cudaStream_t)stream;
        size_t lb = (size_t)c->g.V * 4 * 9 * sizeof(double2);
        c->U64.alloc(lb);
        c->U32.alloc((size_t)c->g.V * 4 * 6 * sizeof(float2));
        DWF_CUDA(cudaMemcpyAsync(c->U64.p, links, lb, is_device_ptr(links) ? cudaMemcpyDeviceToDevice
                                                                             : cudaMemcpyHostToDevice,
                                 c->stream));
        dwf::pack_links(c, c->U64.as<double2>());
        c->scal.alloc(sizeof(double) * dwf::NSCALAR);
        DWF_CUDA(cudaMemsetAsync(c->scal.p, 0, c->scal.bytes, c->stream));
        DWF_CUDA(cudaMallocHost((void **)&c->hscal, sizeof(double) * dwf::NSCALAR));
        c->red_part.alloc(sizeof(double2) * 1024 * 8);
        c->red_count.alloc(sizeof(unsigned));
        DWF_CUDA(cudaMemsetAsync(c->red_count.p, 0, sizeof(unsigned), c->stream));
        DWF_CUDA(cudaStreamSynchronize(c->stream));
        return DWF_OK;
    });
    if (st != DWF_OK) {
        dwf_destroy(c);
        return st;
    }
    *out = c;
    return DWF_OK;
}

}  // namespace dwf

extern "C" {

dwf_status dwf_create(dwf_ctx **out, int nlat, const int (*dims)[4], int Ls, double M5, double mf,
                      const void *const *links, int antiperiodic_t, void *stream) {
    if (!out || !dims || !links || nlat < 1 || nlat > 64) return DWF_EINVAL;
    *out = nullptr;
    if (nlat == 1) return dwf::create_one(out, dims[0], Ls, M5, mf, links[0], antiperiodic_t, stream);
    return dwf::create_batch(out, nlat, dims, Ls, M5, mf, links, antiperiodic_t, stream);
}

dwf_status dwf_lattice(dwf_ctx *c, int i, dwf_ctx **out) {
    if (!c || !out) return DWF_EINVAL;
    *out = nullptr;
    if (c->members.empty()) {
        if (i != 0) return DWF_EINVAL;
        *out = c;
        return DWF_OK;
    }
    if (i < 0 || i >= (int)c->members.size()) return DWF_EINVAL;
    *out = c->members[i];
    return DWF_OK;
}

void dwf_destroy(dwf_ctx *c) {
    if (!c) return;
    if (!c->members.empty()) {
        dwf::destroy_batch(c);
        return;
    }
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    dwf::prof_reset(c);
    for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
    dwf::mg_free(c);
    if (c->hscal) cudaFreeHost(c->hscal);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

dwf_status dwf_apply(dwf_ctx *c, void *out, const void *in, dwf_prec prec, int dagger, int nrhs) {
    if (!c || !out || !in || nrhs < 1 || nrhs > 65535) return DWF_EINVAL;
    if (prec != DWF_F64 && prec != DWF_F32) return DWF_EINVAL;
    if (out == in) return DWF_EINVAL;
    if (!c->members.empty())
        return dwf::batch_async(c, [&](dwf_ctx *m, size_t off) {
            const size_t e = prec == DWF_F64 ? 16 : 8;
            return dwf_apply(m, (char *)out + off * e, (const char *)in + off * e, prec, dagger, nrhs);
        }, nrhs);
    return guarded(c, [&]() -> dwf_status {
        if (prec == DWF_F64)
            dwf::dslash(c, (double2 *)out, (const double2 *)in, dagger != 0, nrhs);
        else
            dwf::dslash(c, (float2 *)out, (const float2 *)in, dagger != 0, nrhs);
        return DWF_OK;
    });
}

dwf_status dwf_pack(dwf_ctx *c, void *internal, const void *canonical, dwf_prec prec, int nrhs) {
    if (!c || !internal || !canonical || nrhs < 1) return DWF_EINVAL;
    if (prec != DWF_F64 && prec != DWF_F32) return DWF_EINVAL;
    if (!c->members.empty())
        return dwf::batch_async(c, [&](dwf_ctx *m, size_t off) {
            const size_t e = prec == DWF_F64 ? 16 : 8;
            return dwf_pack(m, (char *)internal + off * e, (const char *)canonical + off * 16, prec, nrhs);
        }, nrhs);
    return guarded(c, [&]() -> dwf_status {
        dwf::pack(c, internal, (const double2 *)canonical, prec, nrhs);
        return DWF_OK;
    });
}

dwf_status dwf_unpack(dwf_ctx *c, void *canonical, const void *internal, dwf_prec prec, int nrhs) {
    if (!c || !internal || !canonical || nrhs < 1) return DWF_EINVAL;
    if (prec != DWF_F64 && prec != DWF_F32) return DWF_EINVAL;
    if (!c->members.empty())
        return dwf::batch_async(c, [&](dwf_ctx *m, size_t off) {
            const size_t e = prec == DWF_F64 ? 16 : 8;
            return dwf_unpack(m, (char *)canonical + off * 16, (const char *)internal + off * e, prec, nrhs);
        }, nrhs);
    return guarded(c, [&]() -> dwf_status {
        dwf::unpack(c, (double2 *)canonical, internal, prec, nrhs);
        return DWF_OK;
    });
}

dwf_status mg_setup(dwf_ctx *c, int levels, const int *nvec, const int (*block)[4], const mg_params *opt,
                    const void *start) {
    if (!c || levels < 2 || levels > 4 || !nvec || !block) return DWF_EINVAL;
    if (!c->members.empty()) {
        mg_params p;
        if (opt) p = *opt;
        else mg_default_params(&p);
        const int nad = p.split ? nvec[0] / 2 : nvec[0];
        const bool host = start && !is_device_ptr(start);
        return dwf::batch_sync(c, [&](dwf_ctx *m, size_t off) {
            return mg_setup(m, levels, nvec, block, &p, start ? (const char *)start + off * 16 : nullptr);
        }, nad, host);
    }
    return guarded(c, [&]() -> dwf_status {
        mg_params p;
        if (opt) p = *opt;
        else mg_default_params(&p);
        return dwf::mg_setup_impl(c, levels, nvec, block, p, start, start && !is_device_ptr(start));
    });
}

dwf_status mg_solve(dwf_ctx *c, const void *b, void *x, double tol, int nrhs, mg_stats *stats) {
    if (!c || !b || !x || nrhs < 1 || !(tol > 0.0)) return DWF_EINVAL;
    if (!c->members.empty()) return dwf::batch_solve(c, b, x, tol, nrhs, stats, !is_device_ptr(b) || !is_device_ptr(x));
    return guarded(c, [&]() -> dwf_status {
        bool host = !is_device_ptr(b) || !is_device_ptr(x);
        return dwf::mg_solve_impl(c, b, x, tol, nrhs, stats, host);
    });
}

dwf_status dwf_cg_solve(dwf_ctx *c, const void *b, void *x, double tol, int maxiter, int nrhs, dwf_prec prec,
                        mg_stats *stats) {
    if (!c || !b || !x || nrhs < 1 || !(tol > 0.0) || maxiter < 1) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status {
        bool host = !is_device_ptr(b) || !is_device_ptr(x);
        return dwf::cg_solve_impl(c, b, x, tol, maxiter, nrhs, prec, stats, host);
    });
}

dwf_status mg_level_info(dwf_ctx *c, int level, int dims_out[4], int *ncomp_out) {
    if (!c || !dims_out || !ncomp_out) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status { dwf::mg_level_info_impl(c, level, dims_out, ncomp_out); return DWF_OK; });
}

dwf_status mg_get_vectors(dwf_ctx *c, int level, void *out) {
    if (!c || !out) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status { dwf::mg_get_vectors_impl(c, level, (double2 *)out); return DWF_OK; });
}

dwf_status mg_get_coarse_links(dwf_ctx *c, int level, void *out) {
    if (!c || !out) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status { dwf::mg_get_coarse_links_impl(c, level, (double2 *)out); return DWF_OK; });
}

dwf_status mg_restrict(dwf_ctx *c, int level, void *cout, const void *fin) {
    if (!c || !cout || !fin) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status { dwf::mg_restrict_impl(c, level, (double2 *)cout, (const double2 *)fin); return DWF_OK; });
}

dwf_status mg_prolong(dwf_ctx *c, int level, void *fout, const void *cin) {
    if (!c || !fout || !cin) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status { dwf::mg_prolong_impl(c, level, (double2 *)fout, (const double2 *)cin); return DWF_OK; });
}

dwf_status mg_coarse_apply(dwf_ctx *c, int level, void *out, const void *in, int dagger, dwf_prec prec) {
    if (!c || !out || !in || out == in) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status { dwf::mg_coarse_apply_impl(c, level, out, in, dagger != 0, prec); return DWF_OK; });
}

dwf_status mg_coarse_solve(dwf_ctx *c, int level, void *x, const void *b) {
    if (!c || !x || !b || x == b) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status { dwf::mg_coarse_solve_impl(c, level, x, b); return DWF_OK; });
}

dwf_status mg_coarse_solve_static(dwf_ctx *c, int level, void *x, const void *b) {
    if (!c || !x || !b || x == b) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status { dwf::mg_coarse_solve_static_impl(c, level, x, b); return DWF_OK; });
}

dwf_status mg_vcycle(dwf_ctx *c, void *x, const void *b) {
    if (!c || !x || !b || x == b) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status { dwf::mg_vcycle_impl(c, (double2 *)x, (const double2 *)b, 1); return DWF_OK; });
}

dwf_status dwf_lowest_modes(dwf_ctx *c, int k, int max_iters, double tol, unsigned int seed, double *evals,
                            void *evecs_dev, double *resid, int *iters) {
    if (!c || !evals || !evecs_dev) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status {
        dwf::lowest_modes_impl(c, k, max_iters, tol, seed, evals, (double2 *)evecs_dev, resid, iters);
        return DWF_OK;
    });
}

dwf_status mg_coarse_overlap(dwf_ctx *c, int level, const void *fields_dev, int nfields, double *overlap) {
    if (!c || !fields_dev || !overlap || nfields < 1) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status {
        dwf::coarse_overlap_impl(c, level, (const double2 *)fields_dev, nfields, overlap);
        return DWF_OK;
    });
}

dwf_status mg_get_adaptive_vectors(dwf_ctx *c, int level, void *out_dev) {
    if (!c || !out_dev || level < 0) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status {
        dwf::mg_get_adaptive_impl(c, level, (double2 *)out_dev);
        return DWF_OK;
    });
}

dwf_status mg_vcycle_batch(dwf_ctx *c, void *x, const void *b, int nrhs) {
    if (!c || !x || !b || x == b || nrhs < 1) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status {
        dwf::mg_vcycle_impl(c, (double2 *)x, (const double2 *)b, nrhs);
        return DWF_OK;
    });
}

const char *dwf_last_error(void) { return dwf::last_error(); }

dwf_status dwf_profile(dwf_ctx *c, int enable) {
    if (!c) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status {
        DWF_CUDA(cudaStreamSynchronize(c->stream));
        dwf::prof_reset(c);
        c->prof = enable != 0;
        return DWF_OK;
    });
}

dwf_status dwf_profile_read(dwf_ctx *c, int kernel_class, long long *launches, double *total_ms) {
    if (!c || !launches || !total_ms || kernel_class < 0 || kernel_class >= dwf::K_NCLASS) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status {
        DWF_CUDA(cudaStreamSynchronize(c->stream));
        long long n = 0;
        double ms = 0.0;
        for (auto &r : c->prof_rec)
            if (r.cls == kernel_class) {
                float t = r.ms;
                if (r.a) DWF_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
                ms += t;
                ++n;
            }
        *launches = n;
        *total_ms = ms;
        return DWF_OK;
    });
}

dwf_status dwf_profile_units(dwf_ctx *c, int kernel_class, long long *units) {
    if (!c || !units || kernel_class < 0 || kernel_class >= dwf::K_NCLASS || !c->members.empty()) return DWF_EINVAL;
    long long u = 0;
    for (auto &r : c->prof_rec)
        if (r.cls == kernel_class) u += r.units;
    *units = u;
    return DWF_OK;
}

unsigned long long dwf_launch_count(void) { return dwf::launch_count(); }

// ---- learned near-null proposal (include/dwfnet.h) ----

dwf_status net_create(dwf_ctx *c, const dwf_net_shape *shape, dwf_net **out) {
    if (!c || !shape || !out) return DWF_EINVAL;
    *out = nullptr;
    return guarded(c, [&]() -> dwf_status {
        *out = dwf::net_create_impl(c, *shape);
        return DWF_OK;
    });
}

dwf_status net_num_params(const dwf_net *net, long long *count) {
    if (!net || !count) return DWF_EINVAL;
    *count = dwf::net_nparams(net);
    return DWF_OK;
}

dwf_status net_set_params(dwf_net *net, const void *params) {
    if (!net || !params) return DWF_EINVAL;
    return guarded(nullptr, [&]() -> dwf_status {
        dwf::net_set_params_impl(net, params, is_device_ptr(params));
        return DWF_OK;
    });
}

dwf_status net_get_params(dwf_net *net, void *params) {
    if (!net || !params) return DWF_EINVAL;
    return guarded(nullptr, [&]() -> dwf_status {
        dwf::net_get_params_impl(net, params, is_device_ptr(params));
        return DWF_OK;
    });
}

dwf_status net_forward(dwf_net *net, dwf_ctx *c, const void *input, unsigned int seed, void *out) {
    if (!net || !c || !out) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status {
        dwf::net_forward_impl(net, c, input, input && is_device_ptr(input), seed, (double2 *)out);
        return DWF_OK;
    });
}

dwf_status net_loss_grad(dwf_net *net, dwf_ctx *c, const void *input, unsigned int seed, const void *targets, int nt,
                         const int block[4], double *loss, void *grad) {
    if (!net || !c || !targets || !block || !loss || nt < 1) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status {
        *loss = dwf::net_loss_grad_impl(net, c, input, input && is_device_ptr(input), seed, (const double2 *)targets,
                                        nt, block, grad, grad && is_device_ptr(grad));
        return DWF_OK;
    });
}

dwf_status net_set_weight_precision(dwf_net *net, dwf_prec prec) {
    if (!net) return DWF_EINVAL;
    return guarded(nullptr, [&]() -> dwf_status {
        dwf::net_set_wprec_impl(net, prec);
        return DWF_OK;
    });
}

dwf_status net_adam(dwf_net *net, double lr, double beta1, double beta2, double eps) {
    if (!net) return DWF_EINVAL;
    return guarded(nullptr, [&]() -> dwf_status {
        dwf::net_adam_impl(net, lr, beta1, beta2, eps);
        return DWF_OK;
    });
}

void net_destroy(dwf_net *net) {
    if (net) dwf::net_free(net);
}

dwf_status net_refine(dwf_net *net, dwf_ctx *c, const void *in_dev, int nfields, void *out_dev) {
    if (!net || !c || !in_dev || !out_dev || nfields < 1) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status {
        dwf::net_refine_impl(net, c, (const double2 *)in_dev, nfields, (double2 *)out_dev);
        return DWF_OK;
    });
}

dwf_status net_refine_loss_grad(dwf_net *net, dwf_ctx *c, const void *in_dev, int nfields, const void *targets,
                                int nt, const int block[4], double *loss, void *grad) {
    if (!net || !c || !in_dev || !targets || !block || !loss || nfields < 1 || nt < 1) return DWF_EINVAL;
    return guarded(c, [&]() -> dwf_status {
        *loss = dwf::net_refine_loss_grad_impl(net, c, (const double2 *)in_dev, nfields, (const double2 *)targets, nt,
                                               block, grad, grad && is_device_ptr(grad));
        return DWF_OK;
    });
}

dwf_status mg_setup_learned(dwf_ctx *c, dwf_net *net, unsigned int seed, int levels, const int *nvec,
                            const int (*block)[4], const mg_params *opt, int pre_iters0, int fallback_iters0,
                            double probe_tol, int probe_max_iters, int *used_fallback) {
    if (!c || !net || !nvec || !block || levels < 2 || pre_iters0 < 0) return DWF_EINVAL;
    if (!c->members.empty()) return DWF_EINVAL;  // one lattice at a time (dwf_lattice)
    if (used_fallback) *used_fallback = 0;
    mg_params p;
    if (opt) p = *opt;
    else mg_default_params(&p);
    const int nad = p.split ? nvec[0] / 2 : nvec[0];
    const bool refiner = dwf::net_is_refiner(net);
    if (!refiner && dwf::net_nout(net) != nad) return DWF_EINVAL;
    dwf::DevBuf start, pre;
    dwf_status s = DWF_OK;
    if (refiner) {
        // a short relaxation from random vectors, then the network refines them
        mg_params p0 = p;
        p0.setup_iters0 = pre_iters0;
        p0.setup_sweeps = 0;
        s = mg_setup(c, levels, nvec, block, &p0, nullptr);
        if (s != DWF_OK) return s;
    }
    s = guarded(c, [&]() -> dwf_status {
        const size_t fb = sizeof(double2) * (size_t)nad * c->g.V * 12 * c->g.Ls;
        start.alloc(fb);
        if (refiner) {
            pre.alloc(fb);
            dwf::mg_get_adaptive_impl(c, 0, pre.as<double2>());
            dwf::net_refine_impl(net, c, pre.as<double2>(), nad, start.as<double2>());
        } else {
            dwf::net_forward_impl(net, c, nullptr, false, seed, start.as<double2>());
        }
        return DWF_OK;
    });
    pre.release();
    if (s != DWF_OK) return s;
    s = mg_setup(c, levels, nvec, block, &p, start.p);
    start.release();
    if (s != DWF_OK || probe_max_iters <= 0) return s;
    const int64_t n = c->g.V * 12 * c->g.Ls;
    dwf::DevBuf b, x;
    s = guarded(c, [&]() -> dwf_status {
        b.alloc(sizeof(double2) * n);
        x.alloc(sizeof(double2) * n);
        dwf::gauss_fill<double2>(c, b.as<double2>(), 1, n, c->g.Ls, c->g.V, false, seed, 3u);
        dwf::bzero<double2>(c, x.as<double2>(), n);
        return DWF_OK;
    });
    if (s != DWF_OK) return s;
    mg_stats st;
    dwf_status ps = mg_solve(c, b.p, x.p, probe_tol, 1, &st);
    if (ps == DWF_OK && st.iters <= probe_max_iters) return DWF_OK;
    if (ps != DWF_OK && ps != DWF_ENOCONV && ps != DWF_EBREAKDOWN) return ps;
    if (used_fallback) *used_fallback = 1;
    p.setup_iters0 = fallback_iters0;
    return mg_setup(c, levels, nvec, block, &p, nullptr);
}

}  // extern "C"
