// Autotuner: times the context's own operations with CUDA events for each
// admissible value of the launch parameters that do not change any result
// (which columns share an FFT CTA, how the slab-solve factor ring divides
// shared memory and whether the right-hand sides stay in it, how many map
// stages the recurrence keeps in flight) and keeps the fastest.  Every
// candidate computes each output with the same arithmetic in the same order,
// so tuned and untuned solves agree bit for bit.
#include <algorithm>
#include <vector>

#include "lss_common.cuh"
#include "lss_ctx.h"

namespace {

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

// Mean milliseconds of fn over reps runs after one untimed run (which also
// builds any table the candidate needs); a negative value if fn failed.
template <typename F>
float time_ms(Timer& t, cudaStream_t s, int reps, F fn) {
    auto refused = [] {
        cudaGetLastError();   // a refused launch must not fail the next candidate
        return -1.0f;
    };
    if (fn()) return refused();
    cudaEventRecord(t.a, s);
    for (int k = 0; k < reps; ++k)
        if (fn()) return refused();
    cudaEventRecord(t.b, s);
    if (cudaEventSynchronize(t.b) != cudaSuccess) return refused();
    float ms = 0;
    cudaEventElapsedTime(&ms, t.a, t.b);
    return ms / reps;
}

int tune_one(lss_ctx* c, int R, cudaStream_t s) {
    const size_t bytes = (size_t)R * c->n * c->n * sizeof(double2);
    double2* x = nullptr;
    double2* y = nullptr;
    cudaError_t e = cudaMalloc(&x, bytes);
    if (!e) e = cudaMalloc(&y, bytes);
    if (!e) e = cudaMemsetAsync(x, 0, bytes, s);
    if (e) {
        if (x) cudaFree(x);
        cudaGetLastError();
        return lss_check_cuda(c, e, "autotune buffers");
    }
    Timer t;
    const std::string err0 = c->err;
    const lss_ctx::Tune keep = c->tune;
    // FFT column group: the LS operator alone
    {
        float best = -1;
        int pick = 0;
        for (int C : lss_fft_col_candidates(c)) {
            c->tune.fft_C = C;
            const float ms = time_ms(t, s, 5, [&] { return lss_matvec(c, x, y, R, MV_IN_MU, MV_OUT_A, nullptr, nullptr, s); });
            if (ms > 0 && (best < 0 || ms < best)) { best = ms; pick = C; }
        }
        c->tune.fft_C = pick ? pick : keep.fft_C;
    }
    // slab-solve plan, then the recurrence ring: one preconditioner apply
    auto sweep = [&] { return lss_sweep(c, x, y, R, s); };
    {
        float best = -1;
        lss_ctx::Tune pick = c->tune;
        for (int nr : {1, 2})
            for (int half : {0, 1})
                for (int bsm : {-1, 0})
                    for (int nst : {0, 2, 3, 4}) {
                        if (nr == 2 && (R < 2 || half)) continue;   // two right-hand sides need the whole budget
                        c->tune.solve_nr = nr;
                        c->tune.solve_half = half;
                        c->tune.solve_bsm = bsm;
                        c->tune.solve_nst = nst;
                        const float ms = time_ms(t, s, 3, sweep);
                        if (ms > 0 && (best < 0 || ms < best)) { best = ms; pick = c->tune; }
                    }
        c->tune = pick;
    }
    {   // ring stages of the 32-wide slabs' own launches (they set each pass's critical path)
        bool wide = false;
        for (const auto& sd : c->slabs) wide |= sd.ldw == 32;
        bool narrow = false;
        for (const auto& sd : c->slabs) narrow |= sd.ldw == 16;
        if (wide && narrow) {
            float best = -1;
            int pick = 0;
            for (int nst : {0, 2, 3, 4}) {
                c->tune.solve_nst_w = nst;
                const float ms = time_ms(t, s, 3, sweep);
                if (ms > 0 && (best < 0 || ms < best)) { best = ms; pick = nst; }
            }
            c->tune.solve_nst_w = pick;
        }
    }
    {
        float best = -1;
        int pick = c->tune.rec_nb;
        for (int nb : {2, 3, 4}) {
            c->tune.rec_nb = nb;
            const float ms = time_ms(t, s, 3, sweep);
            if (ms > 0 && (best < 0 || ms < best)) { best = ms; pick = nb; }
        }
        c->tune.rec_nb = pick;
    }
    cudaStreamSynchronize(s);
    cudaFree(x);
    cudaFree(y);
    cudaGetLastError();   // a refused candidate leaves no error behind
    c->err = err0;
    ++c->buf_gen;         // captured iterations used the old launch parameters
    // tables of every plan the entry points may now use (the fixed-scratch
    // slab operator must not build one later)
    int rc = lss_prepare_solve_tables(c, s);
    if (!rc) rc = lss_check_device_err(c, s);
    return rc;
}

}  // namespace

extern "C" int lss_autotune(lss_ctx* c, int R, int* chosen, void* stream) {
    if (!c) return LSS_ERR_ARG;
    if (R < 1) return lss_fail(c, LSS_ERR_ARG, "autotune: R must be positive");
    if (!c->factored) return lss_fail(c, LSS_ERR_STATE, "autotune before lss_factor");
    if (c->dim == 3) return lss_fail(c, LSS_ERR_UNSUPPORTED, "autotune: 2D grids only");
    cudaStream_t s = (cudaStream_t)stream;
    for (lss_ctx* ci : c->inst) {
        const int rc = lss_autotune(ci, R, nullptr, s);
        if (rc) return lss_fail(c, rc, ci->err);
    }
    if (c->inst.empty()) {
        const int rc = tune_one(c, R, s);
        if (rc) return rc;
    }
    if (chosen) {
        const lss_ctx::Tune& t = c->inst.empty() ? c->tune : c->inst[0]->tune;
        chosen[0] = t.fft_C;
        chosen[1] = t.solve_bsm;
        chosen[2] = t.solve_nst;
        chosen[3] = t.rec_nb;
        chosen[4] = t.solve_nst_w;
        chosen[5] = t.solve_half;
        chosen[6] = t.solve_nr;
    }
    return LSS_OK;
}
