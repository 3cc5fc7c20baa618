// Ragged instances: several independent LS problems (different n, omega and
// medium) behind one context.  Each instance is a full context of its own
// with its own CUDA stream.  A batch call forks the caller's stream into the
// instance streams, drives each instance from a host worker thread (the
// GMRES iteration of an instance waits on its own stream only, so small
// instances keep the GPU busy while others synchronise), and joins the
// instance streams back into the caller's stream.
//
// Vectors of a batch hold the instances one after another: instance q's
// R x n_q^2 complex values start at element R * (n_0^2 + ... + n_{q-1}^2);
// plane-wave directions (R per instance) and per-RHS statistics are
// instance-major (dirs[(q * R + r) * 2 + a], stats[q * R + r]); a medium
// gradient holds instance q's n_q^2 values at element n_0^2 + ... + n_{q-1}^2.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <functional>
#include <string>
#include <thread>
#include <vector>

#include "lss_common.cuh"
#include "lss_ctx.h"

namespace {

constexpr int kMaxWorkers = 32;   // host threads driving the instances of one call

// Runs fn(q, instance, stream) for every instance, concurrently, between a
// fork from s and a join into s.  Returns the first error other than
// LSS_ERR_NOCONVERGE (lowest instance first), else LSS_ERR_NOCONVERGE if an
// instance did not converge, else LSS_OK; the batch context's message names
// the instance.
int batch_run(lss_ctx* c, cudaStream_t s, const std::function<int(int, lss_ctx*, cudaStream_t)>& fn) {
    const int nq = (int)c->inst.size();
    int rc = lss_check_cuda(c, cudaEventRecord(c->fork_ev, s), "batch fork");
    for (int q = 0; q < nq && !rc; ++q)
        rc = lss_check_cuda(c, cudaStreamWaitEvent(c->inst_stream[q], c->fork_ev, 0), "batch fork");
    if (rc) return rc;
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<int> rcs(nq, LSS_OK);
    std::atomic<int> next{0};
    auto worker = [&]() {
        cudaSetDevice(dev);
        for (int q; (q = next.fetch_add(1)) < nq;) rcs[q] = fn(q, c->inst[q], c->inst_stream[q]);
    };
    const int nw = std::min(nq, kMaxWorkers);
    std::vector<std::thread> pool;
    for (int t = 1; t < nw; ++t) pool.emplace_back(worker);
    worker();
    for (auto& t : pool) t.join();
    for (int q = 0; q < nq; ++q) {
        cudaError_t e = cudaEventRecord(c->inst_done[q], c->inst_stream[q]);
        if (!e) e = cudaStreamWaitEvent(s, c->inst_done[q], 0);
        if (e && !rc) rc = lss_check_cuda(c, e, "batch join");
    }
    if (rc) return rc;
    int first_nc = -1;
    for (int q = 0; q < nq; ++q) {
        if (rcs[q] == LSS_OK) continue;
        if (rcs[q] == LSS_ERR_NOCONVERGE) {
            if (first_nc < 0) first_nc = q;
            continue;
        }
        return lss_fail(c, rcs[q], "instance " + std::to_string(q) + ": " + c->inst[q]->err);
    }
    if (first_nc >= 0)
        return lss_fail(c, LSS_ERR_NOCONVERGE, "instance " + std::to_string(first_nc) + ": " + c->inst[first_nc]->err);
    return LSS_OK;
}

long long off(const lss_ctx* c, int q, int R) { return (long long)R * c->inst_off[q]; }

}  // namespace

// One host thread issues every instance's launches, each on its own stream,
// between a fork from s and a join into s (no host synchronisation inside: the
// lockstep Krylov driver calls this once per iteration).
int lss_batch_op(lss_ctx* c, int which, const double2* x, double2* y, int R, int transpose, cudaStream_t s) {
    const int nq = (int)c->inst.size();
    int rc = lss_check_cuda(c, cudaEventRecord(c->fork_ev, s), "batch fork");
    for (int q = 0; q < nq && !rc; ++q) {
        lss_ctx* ci = c->inst[q];
        cudaStream_t sq = c->inst_stream[q];
        rc = lss_check_cuda(c, cudaStreamWaitEvent(sq, c->fork_ev, 0), "batch fork");
        if (rc) break;
        const long long o = off(c, q, R);
        if (which == 0)
            rc = lss_matvec(ci, x + o, y + o, R, transpose ? MV_IN_U : MV_IN_MU, transpose ? MV_OUT_AT : MV_OUT_A,
                            nullptr, nullptr, sq);
        else
            rc = transpose ? lss_sweep_t(ci, x + o, y + o, R, sq) : lss_sweep(ci, x + o, y + o, R, sq);
        if (rc) rc = lss_fail(c, rc, "instance " + std::to_string(q) + ": " + ci->err);
        cudaError_t e = cudaEventRecord(c->inst_done[q], sq);
        if (!e) e = cudaStreamWaitEvent(s, c->inst_done[q], 0);
        if (e && !rc) rc = lss_check_cuda(c, e, "batch join");
    }
    return rc;
}

void lss_batch_free(lss_ctx* c) {
    for (lss_ctx* ci : c->inst)
        if (ci) lss_destroy(ci);
    for (cudaStream_t st : c->inst_stream)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : c->inst_done)
        if (e) cudaEventDestroy(e);
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    c->inst.clear();
    c->inst_stream.clear();
    c->inst_done.clear();
}

int lss_batch_factor(lss_ctx* c, cudaStream_t s) {
    int rc = batch_run(c, s, [](int, lss_ctx* ci, cudaStream_t sq) { return lss_factor(ci, sq); });
    if (!rc) rc = lss_check_cuda(c, cudaStreamSynchronize(s), "batch factor");
    c->factored = rc == LSS_OK;
    return rc;
}

int lss_batch_plane_wave_rhs(lss_ctx* c, const double* dirs, int R, double2* g, double2* uI, cudaStream_t s) {
    return batch_run(c, s, [&](int q, lss_ctx* ci, cudaStream_t sq) {
        return lss_plane_wave_rhs(ci, dirs + (size_t)q * R * 2, R, g + off(c, q, R), uI ? uI + off(c, q, R) : nullptr,
                                  sq);
    });
}

int lss_batch_apply(lss_ctx* c, int which, const double2* x, double2* y, int R, int transpose, cudaStream_t s) {
    return batch_run(c, s, [&](int q, lss_ctx* ci, cudaStream_t sq) {
        const long long o = off(c, q, R);
        return which == 0 ? lss_apply_A(ci, x + o, y + o, R, transpose, sq)
                          : lss_apply_P(ci, x + o, y + o, R, transpose, sq);
    });
}

int lss_batch_solve(lss_ctx* c, const double2* g, double2* u, int R, const lss_gmres* o, lss_stats* st,
                    cudaStream_t s, int adjoint) {
    // default: every instance's right-hand sides in one lockstep Krylov
    // iteration; LSS_BATCH_THREADS=1 drives each instance's own solve from a
    // host thread instead
    const char* ev = std::getenv("LSS_BATCH_THREADS");
    if (!(ev && ev[0] == '1')) {
        int rc = LSS_OK;
        if (adjoint)
            rc = batch_run(c, s, [](int, lss_ctx* ci, cudaStream_t sq) { return lss_prepare_sweep_t(ci, sq); });
        return rc ? rc : lss_fgmres_batch(c, g, u, R, o, st, s, adjoint ? 1 : 0);
    }
    return batch_run(c, s, [&](int q, lss_ctx* ci, cudaStream_t sq) {
        const long long v = off(c, q, R);
        lss_stats* sq_st = st ? st + (size_t)q * R : nullptr;
        return adjoint ? lss_adjoint_solve(ci, g + v, u + v, R, o, sq_st, sq)
                       : lss_solve(ci, g + v, u + v, R, o, sq_st, sq);
    });
}

int lss_batch_gradient(lss_ctx* c, const double2* mu, const double2* u, const double* dirs, int R, double* grad,
                       cudaStream_t s) {
    return batch_run(c, s, [&](int q, lss_ctx* ci, cudaStream_t sq) {
        const long long v = off(c, q, R);
        return lss_medium_gradient(ci, mu + v, u + v, dirs + (size_t)q * R * 2, R, grad + c->inst_off[q], sq);
    });
}

extern "C" {

int lss_setup_batch(lss_ctx** out, int n_inst, const lss_grid* g, const double* omega, const double* const* m_dev,
                    const lss_pml* pml, const lss_slab* slab, int precision, void* stream) {
    if (!out) return lss_fail(nullptr, LSS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_inst < 1 || !g || !omega || !m_dev || !pml || !slab)
        return lss_fail(nullptr, LSS_ERR_ARG, "setup_batch: bad arguments");
    for (int q = 0; q < n_inst; ++q)
        if (g[q].dim != 2) return lss_fail(nullptr, LSS_ERR_UNSUPPORTED, "setup_batch: 2D instances only");
    for (int q = 0; q < n_inst; ++q)
        if (!m_dev[q]) return lss_fail(nullptr, LSS_ERR_ARG, "setup_batch: m of instance " + std::to_string(q) + " is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    lss_ctx* c = new lss_ctx();
    c->prec = precision;
    c->fronts = slab->fronts == 2 ? 2 : 1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c->num_sms <= 0)
        c->num_sms = 1;
    c->inst.assign(n_inst, nullptr);
    c->inst_stream.assign(n_inst, nullptr);
    c->inst_done.assign(n_inst, nullptr);
    c->inst_off.assign(n_inst + 1, 0);
    for (int q = 0; q < n_inst; ++q) c->inst_off[q + 1] = c->inst_off[q] + (long long)g[q].n * g[q].n;
    cudaError_t e = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming);
    for (int q = 0; q < n_inst && !e; ++q) {
        e = cudaStreamCreateWithFlags(&c->inst_stream[q], cudaStreamNonBlocking);
        if (!e) e = cudaEventCreateWithFlags(&c->inst_done[q], cudaEventDisableTiming);
    }
    if (e) {
        cudaGetLastError();
        lss_batch_free(c);
        delete c;
        return lss_fail(nullptr, LSS_ERR_CUDA, "setup_batch: streams");
    }
    // the instances' set-ups (host work and their own synchronisation) run
    // concurrently; each thread reports its error text itself
    std::vector<int> rcs(n_inst, LSS_OK);
    std::vector<std::string> msgs(n_inst);
    int rc = batch_run(c, s, [&](int q, lss_ctx*, cudaStream_t sq) {
        lss_ctx* ci = nullptr;
        const int r = lss_setup(&ci, &g[q], omega[q], m_dev[q], pml, slab, precision, sq);
        c->inst[q] = ci;
        rcs[q] = r;
        if (r) msgs[q] = lss_last_error(nullptr);
        return LSS_OK;
    });
    std::string m = rc ? c->err : std::string();
    for (int q = 0; q < n_inst && !rc; ++q)
        if (rcs[q]) {
            rc = rcs[q];
            m = "setup_batch: instance " + std::to_string(q) + ": " + msgs[q];
        }
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) {
        rc = LSS_ERR_CUDA;
        m = std::string("setup_batch: ") + cudaGetErrorString(cudaGetLastError());
    }
    if (rc) {
        lss_batch_free(c);   // destroys the instances that were set up
        delete c;
        return lss_fail(nullptr, rc, m);
    }
    *out = c;
    return LSS_OK;
}

int lss_batch_info(const lss_ctx* c, int* n_inst, long long* elems_per_rhs) {
    if (!c || c->inst.empty()) return LSS_ERR_ARG;
    if (n_inst) *n_inst = (int)c->inst.size();
    if (elems_per_rhs) *elems_per_rhs = c->inst_off.back();
    return LSS_OK;
}

int lss_batch_instance(lss_ctx* c, int q, lss_ctx** inst) {
    if (!c || !inst) return LSS_ERR_ARG;
    if (c->inst.empty() || q < 0 || q >= (int)c->inst.size())
        return lss_fail(c, LSS_ERR_ARG, "batch_instance: not a batch context or index out of range");
    *inst = c->inst[q];
    return LSS_OK;
}

}  // extern "C"
