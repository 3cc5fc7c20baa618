// C ABI entry points (include/lss.h): argument checks, context set-up,
// orchestration of the kernels in the other translation units.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "lss_common.cuh"
#include "lss_ctx.h"
#include "lss3d.h"

namespace {

thread_local std::string g_setup_error;

__global__ void cast_c128_c64(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

void free_ctx(lss_ctx* c) {
    if (!c) return;
    if (!c->inst.empty() || c->fork_ev) lss_batch_free(c);
    if (c->d3) lss3_free(c);
    for (auto& g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);   // refused captures are kept as null entries
    for (auto st : c->aux_stream) cudaStreamDestroy(st);
    for (auto ev : c->aux_event) cudaEventDestroy(ev);
    if (c->fork_event) cudaEventDestroy(c->fork_event);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (auto& r : c->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (auto e : c->iter_ev)
        if (e) cudaEventDestroy(e);
    if (c->host_flags) cudaFreeHost(c->host_flags);
    void* ptrs[] = {c->m, c->khatT, c->tw, c->gam_phys, c->gam_aux, c->gam_aux_r, c->coef64,
                    c->coef == c->coef64 ? nullptr : c->coef, c->fac, c->cr_work, c->iface, c->iface_t, c->d_slabs,
                    c->d_err, c->d_bar, c->mv_buf, c->f_buf, c->side_buf, c->z_buf, c->kr_buf, c->red_buf,
                    c->io_buf, c->dir_buf, c->gr_buf, c->ifx_buf, c->ifp_buf, c->gm_buf, c->hz_buf, c->seg_buf,
                    c->th_buf, c->tq_buf};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (void* p : c->chunk_dev)
        if (p) cudaFree(p);
    delete c;
}

bool is_batch(const lss_ctx* c) { return !c->inst.empty(); }

// Waits on a grid barrier one arrival short of its target and on an mbarrier
// nobody arrives at: both expire after the library's wait limit and set
// LSS_DERR_TIMEOUT; a third wait then returns at once (the flag is set).
__global__ void wait_selftest_kernel(unsigned* counter, int* err) {
    __shared__ uint64_t bar;
    grid_barrier_count(counter, 2u, err);     // one block: the second arrival never comes
    if (threadIdx.x == 0) {
        atomicAnd(err, ~LSS_DERR_TIMEOUT);    // re-arm for the mbarrier wait
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_wait(&bar, 0u, err);             // nothing arrives on phase 0
        grid_barrier_count(counter, 4u, err); // flag set: returns without waiting
    }
}

int batch_only_per_instance(lss_ctx* c, const char* what) {
    return lss_fail(c, LSS_ERR_ARG, std::string(what) + ": not defined on a batch context; call it on an instance "
                                                        "(lss_batch_instance)");
}

int dalloc(lss_ctx* c, void** p, size_t bytes, const char* what) {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return lss_fail(c, LSS_ERR_OOM, std::string("device allocation failed: ") + what);
    }
    return LSS_OK;
}

}  // namespace

// ---------------------------------------------------------------- profiling
namespace {
cudaEvent_t take_event(lss_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

ProfScope::ProfScope(lss_ctx* c_, cudaStream_t s_, int cat_, int n_launch) : c(c_), s(s_), cat(cat_), n(n_launch) {
    c->launches[cat] += n;
    if (c->prof_on) {
        a = take_event(c);
        cudaEventRecord(a, s);
    }
}

ProfScope::~ProfScope() {
    if (c->prof_on && a) {
        cudaEvent_t b = take_event(c);
        cudaEventRecord(b, s);
        c->prof.push_back({cat, a, b, n});
    }
}

std::mutex& lss_config_mutex() {
    static std::mutex m;
    return m;
}

long long& lss_dev_cache(const void* key, int slot) {
    static std::map<std::tuple<const void*, int, int>, long long> cache;   // nodes never move
    int dev = 0;
    cudaGetDevice(&dev);
    return cache[std::make_tuple(key, slot, dev)];
}

// ---------------------------------------------------------------- status helpers
int lss_fail(lss_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    else g_setup_error = msg;
    return code;
}

int lss_check_cuda(lss_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return LSS_OK;
    return lss_fail(c, LSS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int lss_check_device_err(lss_ctx* c, cudaStream_t s) {
    if (!c->d_err) {   // a batch: its instances' status words
        for (size_t q = 0; q < c->inst.size(); ++q) {
            const int rc = lss_check_device_err(c->inst[q], s);
            if (rc) return lss_fail(c, rc, "instance " + std::to_string(q) + ": " + c->inst[q]->err);
        }
        return LSS_OK;
    }
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return lss_check_cuda(c, e, "device status");
    if (!h) return LSS_OK;
    cudaMemsetAsync(c->d_err, 0, sizeof(int), s);
    if (h & LSS_DERR_TIMEOUT) return lss_fail(c, LSS_ERR_TIMEOUT, "a bounded device wait expired");
    if (h & LSS_DERR_SINGULAR) return lss_fail(c, LSS_ERR_SINGULAR, "zero or non-finite pivot in a slab factor");
    return lss_fail(c, LSS_ERR_CUDA, "device error word set");
}

int lss_grow(lss_ctx* c, void** p, size_t* cap, size_t bytes) {
    if (bytes <= *cap && *p) return LSS_OK;
    ++c->buf_gen;   // captured graphs that point into the old buffer are stale
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    int rc = dalloc(c, p, bytes, "workspace");
    if (rc) return rc;
    *cap = bytes;
    return LSS_OK;
}

// Medium-dependent part of the set-up: the squared-frequency samples
// [omega^2(1 - max m), omega^2(1 - min m)] (m on I and 0, Sec. 2.3), the
// moving-PML stencils per sample and the slab subproblems.
int lss_set_medium_impl(lss_ctx* c, const double* m_dev, cudaStream_t s) {
    c->factored = false;
    std::vector<double> mh((size_t)c->npts());
    cudaError_t e = cudaMemcpyAsync(c->m, m_dev, mh.size() * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (!e) e = cudaMemcpyAsync(mh.data(), m_dev, mh.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return lss_check_cuda(c, e, "reading m");
    double mmax = 0.0, mmin = 0.0;
    for (double v : mh) {
        if (!std::isfinite(v) || v >= 1.0) return lss_fail(c, LSS_ERR_ARG, "m must be finite and < 1 (m = 1 - 1/c^2)");
        mmax = std::max(mmax, v);
        mmin = std::min(mmin, v);
    }
    c->ns_eff = (mmax == mmin) ? 1 : c->n_samples;
    c->s_lo = c->omega * c->omega * (1.0 - mmax);
    c->s_hi = c->omega * c->omega * (1.0 - mmin);
    if (c->dim == 3) return lss3_set_medium(c, s);
    int rc = lss_build_gamma_aux(c, s);
    if (!rc) rc = lss_assemble_slabs(c, s);
    if (!rc && c->prec == LSS_MIXED) {
        ProfScope ps(c, s, LSS_PROF_SETUP, 1);
        cast_c128_c64<<<4 * c->num_sms, 256, 0, s>>>(c->coef64, (float2*)c->coef, c->coef_len);
        rc = lss_check_cuda(c, cudaGetLastError(), "cast");
    }
    return rc;
}

// ---------------------------------------------------------------- entry points
extern "C" {

int lss_setup(lss_ctx** out, const lss_grid* g, double omega, const double* m_dev, const lss_pml* pml,
              const lss_slab* slab, int precision, void* stream) {
    if (!out) return lss_fail(nullptr, LSS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!g || !m_dev || !pml || !slab) return lss_fail(nullptr, LSS_ERR_ARG, "NULL argument");
    if (g->dim != 2 && g->dim != 3) return lss_fail(nullptr, LSS_ERR_ARG, "dim must be 2 or 3");
    if (g->dim == 2 && (g->n < 4 || g->n > 2048))
        return lss_fail(nullptr, LSS_ERR_UNSUPPORTED, "n must be in [4, 2048]");
    if (g->dim == 3 && (g->n < 3 || g->n > 128))
        return lss_fail(nullptr, LSS_ERR_UNSUPPORTED, "3D: n must be in [3, 128]");
    if (!(omega > 0) || !std::isfinite(omega)) return lss_fail(nullptr, LSS_ERR_ARG, "omega must be positive");
    if (pml->b_pml < 1 || !(pml->C > 0)) return lss_fail(nullptr, LSS_ERR_ARG, "b_pml >= 1 and C > 0 required");
    if (slab->b_slab < 1 || slab->b_aux < 0 || slab->n_samples < 0 || slab->fronts < 0 || slab->fronts > 2 ||
        slab->recursive < 0 || slab->recursive > 1)
        return lss_fail(nullptr, LSS_ERR_ARG, "bad slab parameters");
    if (slab->recursive && g->dim != 3)
        return lss_fail(nullptr, LSS_ERR_UNSUPPORTED, "the recursive approach is for 3D grids");
    if (precision != LSS_FP64 && precision != LSS_MIXED) return lss_fail(nullptr, LSS_ERR_ARG, "bad precision");
    cudaStream_t s = (cudaStream_t)stream;

    lss_ctx* c = new lss_ctx();
    c->dim = g->dim;
    c->n = g->n;
    c->omega = omega;
    c->h = 1.0 / (g->n + 1);
    c->pml = *pml;
    c->slab = *slab;
    c->prec = precision;
    c->b = pml->b_pml;
    c->b_aux = slab->b_aux ? slab->b_aux : pml->b_pml;
    c->n_samples = slab->n_samples ? slab->n_samples : g->n;
    c->fronts = slab->fronts == 2 ? 2 : 1;
    {   // LSS_SOLVE_NR=2: two right-hand sides per slab-solve CTA from the start (else the autotuner decides)
        const char* v = std::getenv("LSS_SOLVE_NR");
        if (v && v[0] == '2') c->tune.solve_nr = 2;
    }
    c->n_tot = c->n + 2 + 2 * c->b;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (c->num_sms <= 0) c->num_sms = 1;
    c->L = 8;
    c->lgL = 3;
    while (c->L < 2 * c->n - 1) { c->L <<= 1; ++c->lgL; }
    if (c->dim == 3) {   // Sec. 3.1: the same construction on 3D slabs (lss3d.cu)
        int rc = lss3_setup(c, m_dev, s);
        if (!rc) rc = lss_set_medium_impl(c, m_dev, s);
        if (!rc) rc = lss_check_cuda(c, cudaStreamSynchronize(s), "setup");
        if (!rc) rc = lss_check_device_err(c, s);
        if (rc) { std::string m = c->err; free_ctx(c); return lss_fail(nullptr, rc, m); }
        *out = c;
        return LSS_OK;
    }

    // slabs along x1 (Sec. 2.3): first = left PML + b_slab layers, middle b_slab,
    // last = the remaining normal layers + right PML.  One front: every slab but
    // the first is padded on the left.  Two fronts (Sec. 2.4 remark 1): the
    // slabs left of the middle slab on the left, those right of it on the
    // right, the middle slab on both sides.
    const int n = c->n, b = c->b, bs = slab->b_slab;
    const int nl = (n + 2 + bs - 1) / bs;
    c->n_slabs = nl;
    c->mid = (nl - 1) / 2;
    long long coff = 0, foff = 0, woff = 0;
    for (int i = 0; i < nl; ++i) {
        SlabDev sd{};
        if (i == 0) {
            sd.s = -b;
            sd.nl = (nl == 1) ? c->n_tot : b + bs;
        } else {
            sd.s = i * bs;
            sd.nl = (i == nl - 1) ? (n + 2 - i * bs) + b : bs;
        }
        const bool left = c->fronts == 2 ? (i > 0 && i <= c->mid) : i > 0;
        const bool right = c->fronts == 2 && i >= c->mid && i < nl - 1;
        sd.na = left ? c->b_aux : 0;
        sd.nr = right ? c->b_aux : 0;
        sd.ll = sd.na + sd.nl - 1;
        sd.w = sd.na + sd.nl + sd.nr;
        if (sd.w > LSS_WMAX) {
            free_ctx(c);
            return lss_fail(nullptr, LSS_ERR_UNSUPPORTED, "a slab subproblem is wider than 32 layers");
        }
        sd.ldw = sd.w <= 16 ? 16 : 32;
        sd.cstride = (sd.w * 9 + 1) & ~1;
        sd.bs = sd.ldw * sd.ldw;
        sd.coef_off = coff;
        sd.fac_off = foff;
        sd.work_off = woff;
        coff += (long long)sd.cstride * c->n_tot;
        foff += cr_fac_entries(c->n_tot, sd.bs, sd.ldw);
        woff += (long long)sd.bs * cr_work_blocks(c->n_tot);
        c->slabs.push_back(sd);
    }

    const int nc = 2 * b + 1;
    const size_t cs = c->csize();
    int rc = LSS_OK;
    rc = rc ? rc : dalloc(c, (void**)&c->m, (size_t)n * n * sizeof(double), "m");
    rc = rc ? rc : dalloc(c, (void**)&c->tw, (size_t)c->L * sizeof(double2), "twiddles");
    rc = rc ? rc : dalloc(c, (void**)&c->khatT, (size_t)c->L * c->L * sizeof(double2), "kernel transform");
    rc = rc ? rc : dalloc(c, (void**)&c->gam_phys, (size_t)nc * nc * 9 * sizeof(double2), "gamma");
    rc = rc ? rc : dalloc(c, (void**)&c->gam_aux, (size_t)c->n_samples * c->b_aux * nc * 9 * sizeof(double2), "gamma aux");
    if (c->fronts == 2)
        rc = rc ? rc : dalloc(c, (void**)&c->gam_aux_r, (size_t)c->n_samples * c->b_aux * nc * 9 * sizeof(double2),
                              "gamma aux right");
    rc = rc ? rc : dalloc(c, (void**)&c->coef64, (size_t)coff * sizeof(double2), "coefficients");
    if (!rc) {
        if (precision == LSS_FP64) c->coef = c->coef64;
        else rc = dalloc(c, &c->coef, (size_t)coff * cs, "coefficients fp32");
    }
    rc = rc ? rc : dalloc(c, &c->fac, (size_t)foff * cs, "slab factors");
    c->work_len = woff;
    rc = rc ? rc : dalloc(c, &c->cr_work, (size_t)2 * woff * cs, "reduction work");
    // 64 bytes of slack: the recurrence copies 16-byte aligned windows that may
    // end up to 15 bytes past the last map row
    const int nmaps = c->fronts == 2 ? 4 : 3;
    rc = rc ? rc : dalloc(c, &c->iface, (size_t)nmaps * nl * c->n_tot * c->n_tot * cs + 64, "interface maps");
    rc = rc ? rc : dalloc(c, (void**)&c->d_slabs, nl * sizeof(SlabDev), "slabs");
    rc = rc ? rc : dalloc(c, (void**)&c->d_err, sizeof(int), "status");
    rc = rc ? rc : dalloc(c, (void**)&c->d_bar, 2 * sizeof(unsigned), "barrier");
    if (rc) { std::string m = c->err; free_ctx(c); return lss_fail(nullptr, rc, m); }
    cudaMemcpyAsync(c->d_slabs, c->slabs.data(), nl * sizeof(SlabDev), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(c->d_err, 0, sizeof(int), s);
    cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned), s);
    cudaMemsetAsync(c->iface, 0, (size_t)nmaps * nl * c->n_tot * c->n_tot * cs, s);

    c->coef_len = coff;
    rc = lss_fft_configure(c);
    if (!rc) rc = lss_build_kernel(c, s);
    if (!rc) rc = lss_build_interior_stencils(c, s);
    if (!rc) rc = lss_build_gamma_phys(c, s);
    if (!rc) rc = lss_set_medium_impl(c, m_dev, s);
    if (!rc) rc = lss_check_cuda(c, cudaStreamSynchronize(s), "setup");
    if (!rc) rc = lss_check_device_err(c, s);
    if (rc) { std::string m = c->err; free_ctx(c); return lss_fail(nullptr, rc, m); }
    *out = c;
    return LSS_OK;
}

int lss_set_medium(lss_ctx* c, const double* m_dev, void* stream) {
    if (!c) return LSS_ERR_ARG;
    if (is_batch(c)) return batch_only_per_instance(c, "set_medium");
    if (!m_dev) return lss_fail(c, LSS_ERR_ARG, "set_medium: m is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = lss_set_medium_impl(c, m_dev, s);
    if (!rc) rc = lss_check_cuda(c, cudaGetLastError(), "set_medium");
    return rc;
}

int lss_profile(lss_ctx* c, int enable) {
    if (!c) return LSS_ERR_ARG;
    for (lss_ctx* ci : c->inst) lss_profile(ci, enable);
    c->prof_on = enable != 0;
    return LSS_OK;
}

int lss_set_graphs(lss_ctx* c, int enable) {
    if (!c) return LSS_ERR_ARG;
    for (lss_ctx* ci : c->inst) lss_set_graphs(ci, enable);
    c->graphs_on = enable != 0;
    return LSS_OK;
}

int lss_graph_count(const lss_ctx* c, int* captured, int* refused) {
    if (!c) return LSS_ERR_ARG;
    int a = 0, b = 0;
    for (const auto& g : c->graphs) (g.exec ? a : b) += 1;
    for (const lss_ctx* ci : c->inst) {
        int x = 0, y = 0;
        lss_graph_count(ci, &x, &y);
        a += x;
        b += y;
    }
    if (captured) *captured = a;
    if (refused) *refused = b;
    return LSS_OK;
}

int lss_profile_read(lss_ctx* c, double* ms, long long* launches, int ncat) {
    if (!c || ncat < 0) return LSS_ERR_ARG;
    if (is_batch(c)) {   // sums over the instances
        std::vector<double> sm(LSS_PROF_NCAT, 0.0), m1(LSS_PROF_NCAT);
        std::vector<long long> sl(LSS_PROF_NCAT, 0), l1(LSS_PROF_NCAT);
        for (lss_ctx* ci : c->inst) {
            const int rc = lss_profile_read(ci, m1.data(), l1.data(), LSS_PROF_NCAT);
            if (rc) return lss_fail(c, rc, ci->err);
            for (int k = 0; k < LSS_PROF_NCAT; ++k) { sm[k] += m1[k]; sl[k] += l1[k]; }
        }
        for (int k = 0; k < ncat && k < LSS_PROF_NCAT; ++k) {
            if (ms) ms[k] = sm[k];
            if (launches) launches[k] = sl[k];
        }
        return LSS_OK;
    }
    std::vector<double> acc(LSS_PROF_NCAT, 0.0);
    for (auto& r : c->prof) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e) return lss_check_cuda(c, e, "profile");
        float t = 0;
        cudaEventElapsedTime(&t, r.a, r.b);
        acc[r.cat] += t;
        c->ev_pool.push_back(r.a);
        c->ev_pool.push_back(r.b);
    }
    c->prof.clear();
    for (int k = 0; k < ncat && k < LSS_PROF_NCAT; ++k) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = c->launches[k];
    }
    for (int k = 0; k < LSS_PROF_NCAT; ++k) c->launches[k] = 0;
    return LSS_OK;
}

int lss_factor(lss_ctx* c, void* stream) {
    if (!c) return LSS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (is_batch(c)) return lss_batch_factor(c, s);
    c->factored = false;
    int rc = c->dim == 3 ? lss3_factor(c, s) : lss_factor_slabs(c, s);
    if (!rc) rc = lss_check_cuda(c, cudaStreamSynchronize(s), "factor");
    if (!rc) rc = lss_check_device_err(c, s);
    if (rc) return rc;
    c->factored = true;
    return LSS_OK;
}

int lss_plane_wave_rhs(lss_ctx* c, const double* dirs_host, int R, void* g_dev, void* uI_dev, void* stream) {
    if (!c) return LSS_ERR_ARG;
    if (!dirs_host || !g_dev || R < 1) return lss_fail(c, LSS_ERR_ARG, "plane_wave_rhs: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    if (is_batch(c)) return lss_batch_plane_wave_rhs(c, dirs_host, R, (double2*)g_dev, (double2*)uI_dev, s);
    int rc = lss_grow(c, &c->dir_buf, &c->dir_cap, (size_t)R * c->dim * sizeof(double));
    if (rc) return rc;
    rc = lss_check_cuda(c, cudaMemcpyAsync(c->dir_buf, dirs_host, (size_t)R * c->dim * sizeof(double),
                                           cudaMemcpyHostToDevice, s), "directions");
    if (rc) return rc;
    return lss_matvec(c, nullptr, (double2*)g_dev, R, MV_IN_PLANEWAVE, MV_OUT_NEG, (const double*)c->dir_buf,
                      (double2*)uI_dev, s);
}

int lss_apply_A(lss_ctx* c, const void* x, void* y, int R, int transpose, void* stream) {
    if (!c) return LSS_ERR_ARG;
    if (!x || !y || R < 1 || x == y) return lss_fail(c, LSS_ERR_ARG, "apply_A: bad arguments");
    if (is_batch(c)) return lss_batch_apply(c, 0, (const double2*)x, (double2*)y, R, transpose, (cudaStream_t)stream);
    return lss_matvec(c, (const double2*)x, (double2*)y, R, transpose ? MV_IN_U : MV_IN_MU,
                      transpose ? MV_OUT_AT : MV_OUT_A, nullptr, nullptr, (cudaStream_t)stream);
}

int lss_apply_P(lss_ctx* c, const void* x, void* y, int R, int transpose, void* stream) {
    if (!c) return LSS_ERR_ARG;
    if (!x || !y || R < 1) return lss_fail(c, LSS_ERR_ARG, "apply_P: bad arguments");
    if (!c->factored) return lss_fail(c, LSS_ERR_STATE, "apply_P before lss_factor");
    if (is_batch(c)) return lss_batch_apply(c, 1, (const double2*)x, (double2*)y, R, transpose, (cudaStream_t)stream);
    if (transpose && c->dim == 3)
        return lss_fail(c, LSS_ERR_UNSUPPORTED, "apply_P: the transposed sweep is built for 2D grids only");
    if (transpose && c->fronts == 2)
        return lss_fail(c, LSS_ERR_UNSUPPORTED, "apply_P: the transposed sweep is built for one front only");
    if (transpose) return lss_sweep_t(c, (const double2*)x, (double2*)y, R, (cudaStream_t)stream);
    return lss_sweep(c, (const double2*)x, (double2*)y, R, (cudaStream_t)stream);
}

int lss_solve(lss_ctx* c, const void* g, void* u, int R, const lss_gmres* o, lss_stats* stats, void* stream) {
    if (!c) return LSS_ERR_ARG;
    if (!g || !u || !o || R < 1 || g == u) return lss_fail(c, LSS_ERR_ARG, "solve: bad arguments");
    if (o->restart < 1 || o->restart > 200 || !(o->tol > 0) || o->max_iter < 1)
        return lss_fail(c, LSS_ERR_ARG, "solve: bad GMRES options");
    if (!c->factored) return lss_fail(c, LSS_ERR_STATE, "solve before lss_factor");
    if (is_batch(c)) return lss_batch_solve(c, (const double2*)g, (double2*)u, R, o, stats, (cudaStream_t)stream, 0);
    return lss_fgmres(c, (const double2*)g, (double2*)u, R, o, stats, (cudaStream_t)stream);
}

int lss_adjoint_solve(lss_ctx* c, const void* rhs, void* mu, int R, const lss_gmres* o, lss_stats* stats,
                      void* stream) {
    if (!c) return LSS_ERR_ARG;
    if (!rhs || !mu || !o || R < 1 || rhs == mu) return lss_fail(c, LSS_ERR_ARG, "adjoint_solve: bad arguments");
    if (o->restart < 1 || o->restart > 200 || !(o->tol > 0) || o->max_iter < 1)
        return lss_fail(c, LSS_ERR_ARG, "adjoint_solve: bad GMRES options");
    if (!c->factored) return lss_fail(c, LSS_ERR_STATE, "adjoint_solve before lss_factor");
    if (c->dim == 3) return lss_fail(c, LSS_ERR_UNSUPPORTED, "adjoint_solve: 2D grids only");
    if (c->fronts == 2) return lss_fail(c, LSS_ERR_UNSUPPORTED, "adjoint_solve: one sweeping front only");
    if (is_batch(c))
        return lss_batch_solve(c, (const double2*)rhs, (double2*)mu, R, o, stats, (cudaStream_t)stream, 1);
    return lss_fgmres(c, (const double2*)rhs, (double2*)mu, R, o, stats, (cudaStream_t)stream, 1);
}

int lss_helmholtz_solve(lss_ctx* c, const void* f, void* u, int R, const lss_gmres* o, lss_stats* stats,
                        void* stream) {
    if (!c) return LSS_ERR_ARG;
    if (!f || !u || !o || R < 1) return lss_fail(c, LSS_ERR_ARG, "helmholtz_solve: bad arguments");
    if (o->restart < 1 || o->restart > 200 || !(o->tol > 0) || o->max_iter < 1)
        return lss_fail(c, LSS_ERR_ARG, "helmholtz_solve: bad GMRES options");
    if (is_batch(c)) return batch_only_per_instance(c, "helmholtz_solve");
    if (c->dim != 2) return lss_fail(c, LSS_ERR_UNSUPPORTED, "helmholtz_solve: 2D grids only");
    if (!c->factored) return lss_fail(c, LSS_ERR_STATE, "helmholtz_solve before lss_factor");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t G = (size_t)R * c->n_tot * c->n_tot;
    int rc = lss_grow(c, &c->hz_buf, &c->hz_cap, 2 * G * sizeof(double2));
    if (rc) return rc;
    double2* F = (double2*)c->hz_buf;
    double2* U = F + G;
    rc = lss_sparsify_beta(c, (const double2*)f, F, R, s);
    if (!rc) rc = lss_fgmres(c, F, U, R, o, stats, s, 2);
    if (rc && rc != LSS_ERR_NOCONVERGE) return rc;
    const int rc2 = lss_extract_grid(c, U, (double2*)u, R, s);
    return rc2 ? rc2 : rc;
}

int lss_medium_gradient(lss_ctx* c, const void* mu, const void* u, const double* dirs_host, int R, double* grad,
                        void* stream) {
    if (!c) return LSS_ERR_ARG;
    if (!mu || !u || !dirs_host || !grad || R < 1) return lss_fail(c, LSS_ERR_ARG, "medium_gradient: bad arguments");
    if (c->dim == 3) return lss_fail(c, LSS_ERR_UNSUPPORTED, "medium_gradient: 2D grids only");
    if (c->fronts == 2) return lss_fail(c, LSS_ERR_UNSUPPORTED, "medium_gradient: one sweeping front only");
    cudaStream_t s = (cudaStream_t)stream;
    if (is_batch(c)) return lss_batch_gradient(c, (const double2*)mu, (const double2*)u, dirs_host, R, grad, s);
    const size_t bytes = (size_t)R * c->n * c->n * sizeof(double2);
    int rc = lss_grow(c, &c->gr_buf, &c->gr_cap, bytes);
    if (!rc) rc = lss_grow(c, &c->dir_buf, &c->dir_cap, (size_t)R * 2 * sizeof(double));
    if (rc) return rc;
    rc = lss_check_cuda(c, cudaMemcpyAsync(c->dir_buf, dirs_host, (size_t)R * 2 * sizeof(double),
                                           cudaMemcpyHostToDevice, s), "directions");
    if (rc) return rc;
    // -omega^2 K mu, then the pointwise product with the total field
    rc = lss_matvec(c, (const double2*)mu, (double2*)c->gr_buf, R, MV_IN_U, MV_OUT_NEG, nullptr, nullptr, s);
    if (rc) return rc;
    return lss_gradient_m(c, (const double2*)c->gr_buf, (const double2*)u, (const double*)c->dir_buf, grad, R, s);
}

int lss_solve_host(lss_ctx* c, const void* g_host, void* u_host, int R, const lss_gmres* o, lss_stats* stats,
                   void* stream) {
    if (!c) return LSS_ERR_ARG;
    if (!g_host || !u_host || R < 1) return lss_fail(c, LSS_ERR_ARG, "solve_host: bad arguments");
    if (is_batch(c)) return batch_only_per_instance(c, "solve_host");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)R * c->npts() * sizeof(double2);
    int rc = lss_grow(c, &c->io_buf, &c->io_cap, 2 * bytes);
    if (rc) return rc;
    double2* gd = (double2*)c->io_buf;
    double2* ud = gd + (size_t)R * c->npts();
    rc = lss_check_cuda(c, cudaMemcpyAsync(gd, g_host, bytes, cudaMemcpyHostToDevice, s), "solve_host upload");
    if (rc) return rc;
    rc = lss_solve(c, gd, ud, R, o, stats, stream);
    if (rc && rc != LSS_ERR_NOCONVERGE) return rc;
    int rc2 = lss_check_cuda(c, cudaMemcpyAsync(u_host, ud, bytes, cudaMemcpyDeviceToHost, s), "solve_host download");
    if (!rc2) rc2 = lss_check_cuda(c, cudaStreamSynchronize(s), "solve_host");
    return rc2 ? rc2 : rc;
}

int lss_apply_slab(lss_ctx* c, int slab, const void* v, void* w, int R, void* stream) {
    if (!c) return LSS_ERR_ARG;
    if (is_batch(c)) return batch_only_per_instance(c, "apply_slab");
    if (!v || !w || R < 1 || slab < 0 || slab >= c->n_slabs)
        return lss_fail(c, LSS_ERR_ARG, "apply_slab: bad arguments");
    if (!c->factored) return lss_fail(c, LSS_ERR_STATE, "apply_slab before lss_factor");
    return lss_slab_apply(c, slab, (const double2*)v, (double2*)w, R, (cudaStream_t)stream);
}

int lss_info(const lss_ctx* c, int* n_tot, int* n_slabs, int* fft_len) {
    if (!c || is_batch(c)) return LSS_ERR_ARG;
    if (n_tot) *n_tot = c->n_tot;
    if (n_slabs) *n_slabs = c->n_slabs;
    if (fft_len) *fft_len = c->L;
    return LSS_OK;
}

int lss_slab_info(const lss_ctx* c, int slab, int* first_x1, int* n_layers, int* n_aux) {
    if (!c || is_batch(c) || slab < 0 || slab >= c->n_slabs) return LSS_ERR_ARG;
    if (c->dim == 3) {
        const Slab3& sd = c->d3->slabs[slab];
        if (first_x1) *first_x1 = sd.s;
        if (n_layers) *n_layers = sd.nl;
        if (n_aux) *n_aux = sd.na;
        return LSS_OK;
    }
    const SlabDev& sd = c->slabs[slab];
    if (first_x1) *first_x1 = sd.s;
    if (n_layers) *n_layers = sd.nl;
    if (n_aux) *n_aux = sd.na;
    return LSS_OK;
}

int lss_get_stencils(const lss_ctx* c, double* alpha, double* beta) {
    if (!c || is_batch(c) || !alpha || !beta) return LSS_ERR_ARG;
    if (c->dim == 3) return lss3_get_stencils(c, alpha, beta);
    for (int o = 0; o < 9; ++o) {
        alpha[2 * o] = c->alpha[o].real();
        alpha[2 * o + 1] = c->alpha[o].imag();
        beta[2 * o] = c->beta[o].real();
        beta[2 * o + 1] = c->beta[o].imag();
    }
    return LSS_OK;
}

int lss_test_inject(lss_ctx* c, int what, int a, long long b, void* stream) {
    if (!c || is_batch(c)) return LSS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (what == 1) {   // zero the coefficients of block row b of slab a
        if (a < 0 || a >= c->n_slabs || b < 0 || b >= c->n_tot) return lss_fail(c, LSS_ERR_ARG, "test_inject: bad slab/row");
        if (c->dim == 3) {
            const Slab3& sd = c->d3->slabs[a];
            const long long off = sd.cf_off + (b * 3 + 1) * (long long)sd.M * 9, len = (long long)sd.M * 9;
            cudaMemsetAsync(c->d3->coef64 + off, 0, len * sizeof(double2), s);
            if (c->d3->coef != c->d3->coef64) cudaMemsetAsync((float2*)c->d3->coef + off, 0, len * sizeof(float2), s);
        } else {
            const SlabDev& sd = c->slabs[a];
            const long long off = sd.coef_off + b * (long long)sd.cstride, len = sd.cstride;
            cudaMemsetAsync(c->coef64 + off, 0, len * sizeof(double2), s);
            if (c->coef != c->coef64) cudaMemsetAsync((float2*)c->coef + off, 0, len * sizeof(float2), s);
        }
        c->factored = false;
        return lss_check_cuda(c, cudaStreamSynchronize(s), "test_inject");
    }
    if (what == 2) {   // bounded device waits that expire
        unsigned* counter = nullptr;
        int rc = dalloc(c, (void**)&counter, sizeof(unsigned), "test counter");
        if (rc) return rc;
        cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
        wait_selftest_kernel<<<1, 32, 0, s>>>(counter, c->d_err);
        rc = lss_check_cuda(c, cudaStreamSynchronize(s), "wait self-test");
        cudaFree(counter);
        if (rc) return rc;
        return lss_check_device_err(c, s);
    }
    return lss_fail(c, LSS_ERR_ARG, "test_inject: unknown injection");
}

const char* lss_last_error(const lss_ctx* c) { return c ? c->err.c_str() : g_setup_error.c_str(); }

void lss_destroy(lss_ctx* c) { free_ctx(c); }

}  // extern "C"
