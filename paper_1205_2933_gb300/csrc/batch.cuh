// A batch of independent lattices behind one context (dwf_create with
// nlat > 1): member contexts on their own streams, fork/join with the batch
// stream, host threads for the synchronous calls.
#pragma once

#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dwf_internal.cuh"

namespace dwf {

struct CoopGate {
    std::mutex mu;
    cudaEvent_t last = nullptr;
    bool used = false;
};

dwf_status create_one(dwf_ctx **out, const int dims[4], int Ls, double M5, double mf, const void *links,
                      int antiperiodic_t, void *stream);
dwf_status create_batch(dwf_ctx **out, int nlat, const int (*dims)[4], int Ls, double M5, double mf,
                        const void *const *links, int antiperiodic_t, void *stream);
void destroy_batch(dwf_ctx *b);
dwf_status batch_solve(dwf_ctx *b, const void *bsrc, void *x, double tol, int nrhs, mg_stats *stats, bool host);
// every member stream waits for the work queued on the batch stream so far / the batch stream waits for every member
dwf_status batch_fork(dwf_ctx *b);
dwf_status batch_join(dwf_ctx *b);
void set_last_error(const std::string &m);
const char *last_error();

inline int64_t member_field(const dwf_ctx *m) { return m->g.V * 12 * (int64_t)m->g.Ls; }

// f(member, element offset) for each member in turn on its own stream;
// offsets advance by nrhs fields of each member's size.
template <typename F> dwf_status batch_async(dwf_ctx *b, F &&f, int nrhs) {
    dwf_status st = batch_fork(b);
    if (st != DWF_OK) return st;
    size_t off = 0;
    for (dwf_ctx *m : b->members) {
        const dwf_status s = f(m, off);
        if (s != DWF_OK && st == DWF_OK) st = s;
        off += (size_t)member_field(m) * nrhs;
    }
    const dwf_status sj = batch_join(b);
    return st != DWF_OK ? st : sj;
}

// f(member, element offset) for all members at once, one host thread each
// (for the calls that synchronise); the first failing member's status and
// message are returned.
template <typename F> dwf_status batch_sync(dwf_ctx *b, F &&f, int nfields, bool host) {
    (void)host;
    dwf_status st = batch_fork(b);
    if (st != DWF_OK) return st;
    const int n = (int)b->members.size();
    std::vector<dwf_status> res(n, DWF_OK);
    std::vector<std::string> msg(n);
    std::vector<std::thread> th;
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        dwf_ctx *m = b->members[i];
        th.emplace_back([&, i, m, off]() {
            if (cudaSetDevice(m->device) != cudaSuccess) {
                res[i] = DWF_ECUDA;
                msg[i] = "cudaSetDevice failed";
                return;
            }
            res[i] = f(m, off);
            if (res[i] != DWF_OK) msg[i] = last_error();
        });
        off += (size_t)member_field(m) * nfields;
    }
    for (auto &t : th) t.join();
    for (int i = 0; i < n; ++i)
        if (res[i] != DWF_OK) {
            set_last_error("lattice " + std::to_string(i) + ": " + msg[i]);
            st = res[i];
            break;
        }
    const dwf_status sj = batch_join(b);
    return st != DWF_OK ? st : sj;
}

}  // namespace dwf
