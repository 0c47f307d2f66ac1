// Batches of independent lattices (dwf_create with nlat > 1) and the gate
// that serialises the members' cooperative launches.
//
// Each member is an ordinary single-lattice context on a stream of its own,
// so the lattices' kernels overlap on the GPU: small lattices, whose kernels
// fill only part of the SMs, run beside a large one.  The cooperative
// coarsest-level solvers size their grids to the whole GPU and spin on
// grid-wide barriers; two of them resident at once, each waiting for SMs the
// other holds, would never finish, so every cooperative launch of a member
// first waits (on the GPU, through an event) for the previous one of the
// batch to complete.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "batch.cuh"
#include "mg.cuh"

namespace dwf {

cudaError_t coop_launch(dwf_ctx *c, const void *fn, dim3 grid, dim3 block, void **args, size_t smem) {
    if (!c->gate) return cudaLaunchCooperativeKernel(fn, grid, block, args, smem, c->stream);
    std::lock_guard<std::mutex> lock(c->gate->mu);
    cudaError_t e;
    if (c->gate->used && (e = cudaStreamWaitEvent(c->stream, c->gate->last, 0)) != cudaSuccess) return e;
    if ((e = cudaLaunchCooperativeKernel(fn, grid, block, args, smem, c->stream)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(c->gate->last, c->stream)) != cudaSuccess) return e;
    c->gate->used = true;
    return cudaSuccess;
}

namespace {

dwf_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return DWF_OK;
    set_last_error(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? DWF_ENOMEM : DWF_ECUDA;
}

// one event per member plus one for the batch stream
cudaEvent_t batch_event(dwf_ctx *b, int i) { return b->batch_ev[i]; }

}  // namespace

dwf_status batch_fork(dwf_ctx *b) {
    const int n = (int)b->members.size();
    cudaError_t e = cudaEventRecord(batch_event(b, n), b->stream);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->members[i]->stream, batch_event(b, n), 0);
    return cuda_status(e);
}

dwf_status batch_join(dwf_ctx *b) {
    const int n = (int)b->members.size();
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaEventRecord(batch_event(b, i), b->members[i]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, batch_event(b, i), 0);
    }
    return cuda_status(e);
}

dwf_status create_batch(dwf_ctx **out, int nlat, const int (*dims)[4], int Ls, double M5, double mf,
                        const void *const *links, int antiperiodic_t, void *stream) {
    for (int i = 0; i < nlat; ++i) {
        if (!links[i]) return DWF_EINVAL;
        for (int k = 0; k < 4; ++k)
            if (dims[i][k] < 1) return DWF_EINVAL;
    }
    if (Ls < 1 || Ls > 128) return DWF_EINVAL;
    dwf_ctx *b = new dwf_ctx();
    b->stream = (cudaStream_t)stream;
    b->g.Ls = Ls;
    b->M5 = M5;
    b->mf = mf;
    b->gate = new CoopGate();
    dwf_status st = DWF_OK;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->gate->last, cudaEventDisableTiming);
    for (int i = 0; i <= nlat && e == cudaSuccess; ++i) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->batch_ev.push_back(ev);
    }
    st = cuda_status(e);
    // the members copy their links on their own streams: first wait for what the caller queued
    if (st == DWF_OK) st = cuda_status(cudaEventRecord(b->batch_ev[nlat], b->stream));
    for (int i = 0; i < nlat && st == DWF_OK; ++i) {
        cudaStream_t s = nullptr;
        st = cuda_status(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        if (st != DWF_OK) break;
        st = cuda_status(cudaStreamWaitEvent(s, b->batch_ev[nlat], 0));
        dwf_ctx *m = nullptr;
        if (st == DWF_OK) st = create_one(&m, dims[i], Ls, M5, mf, links[i], antiperiodic_t, s);
        if (st != DWF_OK) {
            cudaStreamDestroy(s);
            break;
        }
        m->own_stream = true;
        m->gate = b->gate;
        b->members.push_back(m);
    }
    if (st != DWF_OK || (int)b->members.size() != nlat) {
        if (st == DWF_OK) st = DWF_ECUDA;
        destroy_batch(b);
        return st;
    }
    *out = b;
    return DWF_OK;
}

void destroy_batch(dwf_ctx *b) {
    for (dwf_ctx *m : b->members) dwf_destroy(m);
    b->members.clear();
    for (cudaEvent_t ev : b->batch_ev) cudaEventDestroy(ev);
    b->batch_ev.clear();
    if (b->gate) {
        if (b->gate->last) cudaEventDestroy(b->gate->last);
        delete b->gate;
    }
    delete b;
}

dwf_status batch_solve(dwf_ctx *b, const void *bsrc, void *x, double tol, int nrhs, mg_stats *stats, bool host) {
    const int n = (int)b->members.size();
    std::vector<mg_stats> st(n);
    auto t0 = std::chrono::steady_clock::now();
    const dwf_status s = batch_sync(b, [&](dwf_ctx *m, size_t off) {
        size_t i = std::find(b->members.begin(), b->members.end(), m) - b->members.begin();
        return mg_solve(m, (const char *)bsrc + off * 16, (char *)x + off * 16, tol, nrhs, &st[i]);
    }, nrhs, host);
    if (stats) {
        mg_stats t;
        std::memset(&t, 0, sizeof(t));
        for (const mg_stats &q : st) {
            t.iters += q.iters;
            t.restarts += q.restarts;
            t.fine_applies_f64 += q.fine_applies_f64;
            t.fine_applies_f32 += q.fine_applies_f32;
            for (int l = 0; l < 4; ++l) t.coarse_applies[l] += q.coarse_applies[l];
            t.true_res = std::max(t.true_res, q.true_res);
        }
        t.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        *stats = t;
    }
    return s;
}

}  // namespace dwf
