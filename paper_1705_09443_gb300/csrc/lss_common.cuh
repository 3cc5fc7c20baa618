// Shared device helpers: complex arithmetic over float/double, bounded waits,
// TMA bulk copies with mbarriers, and a bounded grid barrier.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#define LSS_WMAX 32            // widest slab subproblem (layers)
// Every device-side wait gives up after ~2 s, counted in SM clock cycles
// (clock64 is cheap to read; the global timer costs hundreds of cycles).
#define LSS_WAIT_CYCLES 4000000000ll

// Device error word bits (ctx->d_err).
#define LSS_DERR_SINGULAR 1
#define LSS_DERR_TIMEOUT 2
#define LSS_DERR_NONFINITE 4
#define LSS_DERR_CONFIG 8      // a kernel was launched with a configuration it does not handle

// ---------------------------------------------------------------- complex
template <typename T> struct cplx_t;
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<float> { using type = float2; };
template <typename T> using cx = typename cplx_t<T>::type;

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
template <typename C> __host__ __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }

__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double2 a, double2 b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return mk(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator*(float2 a, float2 b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) { return mk(s * a.x, s * a.y); }

__host__ __device__ __forceinline__ double2 conjc(double2 a) { return mk(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 conjc(float2 a) { return mk(a.x, -a.y); }
// acc + a*b  (fused multiply-adds)
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
// acc + conj(a)*b
__device__ __forceinline__ double2 cfma_conj(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cfma_conj(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

template <typename C> __device__ __forceinline__ C to_c(double2 a);
template <> __device__ __forceinline__ double2 to_c<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 to_c<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to_d(double2 a) { return a; }
__device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }

// 1/a for complex a (scaled to avoid overflow)
__device__ __forceinline__ double2 crecip(double2 a) {
    double s = fabs(a.x) + fabs(a.y);
    double ar = a.x / s, ai = a.y / s;
    double d = s * (ar * ar + ai * ai);
    return mk(ar / d, -ai / d);
}
__device__ __forceinline__ float2 crecip(float2 a) {
    float s = fabsf(a.x) + fabsf(a.y);
    float ar = a.x / s, ai = a.y / s;
    float d = s * (ar * ar + ai * ai);
    return mk(ar / d, -ai / d);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------- memory ordering
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded grid barrier for cooperative launches (all blocks co-resident).
// bar[0] = arrival count, bar[1] = generation.  On expiry sets LSS_DERR_TIMEOUT
// and returns; once the flag is set later barriers do not wait.
__device__ __forceinline__ void grid_barrier(unsigned* bar, unsigned nblocks, int* err) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        unsigned gen = ld_acquire_u32(bar + 1);
        __threadfence();
        unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == nblocks - 1) {
            bar[0] = 0;
            __threadfence();
            st_release_u32(bar + 1, gen + 1);
        } else {
            const long long t0 = clock64();
            while (ld_acquire_u32(bar + 1) == gen) {
                if (*(volatile int*)err & LSS_DERR_TIMEOUT) break;
                if (clock64() - t0 > LSS_WAIT_CYCLES) { atomicOr(err, LSS_DERR_TIMEOUT); break; }
            }
        }
    }
    __syncthreads();
}

// Bounded grid barrier on a monotonic arrival counter (zeroed before the
// launch): the n-th barrier of a launch waits until the counter reaches
// n * nblocks.  Each CTA adds with a release reduction and polls with acquire
// loads; the error word and the clock are looked at every 64 polls.  On
// expiry sets LSS_DERR_TIMEOUT and returns; once the flag is set later
// barriers do not wait.
__device__ __forceinline__ void grid_barrier_count(unsigned* count, unsigned target, int* err) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
        const long long t0 = clock64();
        for (unsigned it = 0;; ++it) {
            if (ld_acquire_u32(count) >= target) break;
            if ((it & 63u) == 63u) {
                if (*(volatile int*)err & LSS_DERR_TIMEOUT) break;
                if (clock64() - t0 > LSS_WAIT_CYCLES) { atomicOr(err, LSS_DERR_TIMEOUT); break; }
            }
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- TMA bulk copy + mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- cp.async (one complex entry per copy)
template <typename C>
__device__ __forceinline__ void cp_async_entry(C* dst, const C* src, bool valid) {
    static_assert(sizeof(C) == 8 || sizeof(C) == 16, "complex float or double");
    if constexpr (sizeof(C) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src),
                     "r"(valid ? 8 : 0)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                     "r"(valid ? 16 : 0)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 1D bulk copy global -> shared, completion signalled on the mbarrier.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait on phase `parity`; returns false (and flags the error) on expiry.
__device__ __forceinline__ bool mbar_test(uint32_t a, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}
// Bounded wait on phase `parity`: polls first, starts the clock only when the
// phase is not complete yet; returns false (and flags the error) on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err) {
    const uint32_t a = smem_u32(bar);
    if (mbar_test(a, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_test(a, parity)) return true;
        if (clock64() - t0 > LSS_WAIT_CYCLES) break;
    }
    atomicOr(err, LSS_DERR_TIMEOUT);
    return false;
}
