// Tensor-core update of the 3D pivot-block inversion (mixed precision) after an
// outer panel of up to 64 columns J = [J0, J0 + nbo) has been eliminated:
//     W[i][c] += sum_{kk < nbo} W[i][J0 + kk] T64[kk][c]      (c outside J)
// for every slab, complex FP32, as one real product per 128 x 128 complex tile,
// taken in K chunks of 16 complex columns accumulated in tensor memory:
// A' (128 x 32 per chunk, the panel rows' re/im interleaved, exactly their
// FP32 layout) times B' (32 x 256 per chunk, each T64 entry as the 2 x 2
// block [[re, im], [-im, re]]).  Each operand
// is split into TF32 parts x = big + small (big = x rounded to TF32, small =
// the FP32 remainder) and the product taken as big*big + big*small +
// small*big (3xTF32), which keeps about 22 bits of every product.
//
// Shared-memory operands use the no-swizzle K-major layout of 8-row x 16-byte
// core matrices: element (row, k) of a 32-wide K block sits at byte
// ((row / 8) * 8 + k / 4) * 128 + (row % 8) * 16 + (k % 4) * 4, so core
// matrices adjacent in K are 128 bytes apart and adjacent 8-row groups 1024.
// One thread issues the tcgen05.mma instructions (M = 128, N = 256, K = 8 per
// instruction), tcgen05.commit signals an mbarrier, and the four warps read
// the accumulator rows back with tcgen05.ld for the read-modify-write of W.
#include <algorithm>
#include <cstdint>
#include <cstdlib>

#include "lss_common.cuh"
#include "lss_ctx.h"
#include "lss3d.h"

namespace {

constexpr int kTcNB = 16;                         // panel width (complex columns)
constexpr int kTcK = 2 * kTcNB;                   // real K of one product
constexpr int kTileM = 128, kTileN = 256;         // real tile; 128 complex columns
constexpr int kABytes = kTileM * kTcK * 4;        // 16 KB per operand part
constexpr int kBBytes = kTileN * kTcK * 4;        // 32 KB per operand part
constexpr int kTcSmem = 2 * kABytes + 2 * kBBytes + 1024;
constexpr uint32_t kTmemCols = 256;

__device__ __forceinline__ uint32_t core_off(int row, int k) {
    return (uint32_t)((((row >> 3) * (kTcK / 4) + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2));
}

// Round to TF32 (nearest, ties away) and the FP32 remainder.
__device__ __forceinline__ void split_tf32(float x, float& big, float& small) {
    uint32_t b;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(x));
    big = __uint_as_float(b);
    small = x - big;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    // start address, LBO = 128 B (K-adjacent core matrices), SBO = 1024 B
    // (adjacent 8-row groups), descriptor version 1, no swizzle
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((1024u >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::tf32 instruction descriptor: FP32 accumulator, TF32 A and B, both
// K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTileN >> 3) << 17) |
                            ((uint32_t)(kTileM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Persistent: CTA loops over (slab, row tile, column tile) slots.  128 threads.
__global__ void __launch_bounds__(128) f3_update_tc(const Slab3* __restrict__ slabs, int n_slabs,
                                                     float2* __restrict__ W, const float2* __restrict__ T64, int J0,
                                                     int NO, int Tld, int tmax, int* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* Abig = sm;
    unsigned char* Asml = sm + kABytes;
    unsigned char* Bbig = sm + 2 * kABytes;
    unsigned char* Bsml = sm + 2 * kABytes + kBBytes;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * kABytes + 2 * kBBytes);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * kABytes + 2 * kBBytes + 16);
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    unsigned phase = 0;
    bool ok = true;

    const long long slots = (long long)n_slabs * tmax * tmax;
    for (long long slot = blockIdx.x; slot < slots && ok; slot += gridDim.x) {
        const int slab = (int)(slot / ((long long)tmax * tmax));
        const int rem = (int)(slot % ((long long)tmax * tmax));
        const Slab3 sd = slabs[slab];
        const int M = sd.M;
        if (J0 >= M) continue;
        const int tiles = (M + 127) / 128;
        const int ti = rem / tmax, tj = rem % tmax;
        if (ti >= tiles || tj >= tiles) continue;
        const int nbo = min(NO, M - J0);
        const int i0 = ti * 128, c0 = tj * 128;
        float2* w = W + sd.w_off;
        const float2* t64 = T64 + (long long)slab * NO * Tld;
        const int nk = (nbo + kTcNB - 1) / kTcNB;
        for (int kc = 0; kc < nk && ok; ++kc) {
        const int j0 = J0 + kc * kTcNB, nbp = min(kTcNB, nbo - kc * kTcNB);
        const float2* t = t64 + (long long)kc * kTcNB * Tld;

        // ---- operands into shared memory
        {   // A: row tid of the tile, panel columns j0.. (2 nbp reals, zero beyond)
            const int i = i0 + tid;
            float a[kTcK];
            for (int q = 0; q < kTcNB; ++q) {
                float2 v = make_float2(0.f, 0.f);
                if (i < M && q < nbp) v = w[(long long)i * M + j0 + q];
                a[2 * q] = v.x;
                a[2 * q + 1] = v.y;
            }
            for (int k4 = 0; k4 < kTcK / 4; ++k4) {
                float4 hb, hs;
                split_tf32(a[4 * k4 + 0], hb.x, hs.x);
                split_tf32(a[4 * k4 + 1], hb.y, hs.y);
                split_tf32(a[4 * k4 + 2], hb.z, hs.z);
                split_tf32(a[4 * k4 + 3], hb.w, hs.w);
                *reinterpret_cast<float4*>(Abig + core_off(tid, 4 * k4)) = hb;
                *reinterpret_cast<float4*>(Asml + core_off(tid, 4 * k4)) = hs;
            }
        }
        {   // B^T rows 2c, 2c+1 for complex column c = tid: K entries (2kk, 2kk+1)
            const int c = c0 + tid;
            float r0[kTcK], r1[kTcK];
            for (int q = 0; q < kTcNB; ++q) {
                float2 v = make_float2(0.f, 0.f);
                if (c < M && q < nbp) v = t[(long long)q * Tld + c];
                r0[2 * q] = v.x;
                r0[2 * q + 1] = -v.y;
                r1[2 * q] = v.y;
                r1[2 * q + 1] = v.x;
            }
            for (int k4 = 0; k4 < kTcK / 4; ++k4) {
                float4 b0, s0, b1, s1;
                split_tf32(r0[4 * k4 + 0], b0.x, s0.x);
                split_tf32(r0[4 * k4 + 1], b0.y, s0.y);
                split_tf32(r0[4 * k4 + 2], b0.z, s0.z);
                split_tf32(r0[4 * k4 + 3], b0.w, s0.w);
                split_tf32(r1[4 * k4 + 0], b1.x, s1.x);
                split_tf32(r1[4 * k4 + 1], b1.y, s1.y);
                split_tf32(r1[4 * k4 + 2], b1.z, s1.z);
                split_tf32(r1[4 * k4 + 3], b1.w, s1.w);
                *reinterpret_cast<float4*>(Bbig + core_off(2 * tid, 4 * k4)) = b0;
                *reinterpret_cast<float4*>(Bsml + core_off(2 * tid, 4 * k4)) = s0;
                *reinterpret_cast<float4*>(Bbig + core_off(2 * tid + 1, 4 * k4)) = b1;
                *reinterpret_cast<float4*>(Bsml + core_off(2 * tid + 1, 4 * k4)) = s1;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

        // ---- 3xTF32 product: big*big + big*small + small*big, K = 8 per instruction
        if (tid == 0) {
            const uint32_t ab = smem_u32(Abig), as = smem_u32(Asml), bb = smem_u32(Bbig), bs = smem_u32(Bsml);
            uint32_t acc = kc > 0;
            for (int part = 0; part < 3; ++part) {
                const uint32_t pa = part == 2 ? as : ab;
                const uint32_t pb = part == 1 ? bs : bb;
                for (int ks = 0; ks < kTcK / 8; ++ks) {
                    mma_tf32(tmem, smem_desc(pa + ks * 256), smem_desc(pb + ks * 256), acc);
                    acc = 1;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(bar))
                         : "memory");
        }
        if (!mbar_wait(bar, phase, err)) ok = false;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // the next chunk's operand writes must not overtake this chunk's products
        __syncthreads();
        }   // K chunks
        if (!ok) break;

        // ---- epilogue, 8 chunks of 16 complex columns: each thread moves its
        // accumulator row (tcgen05.ld) into shared memory (row stride 33
        // floats, no bank conflicts), then the CTA adds the chunk to W with
        // consecutive threads on consecutive columns of a row
        float* S = reinterpret_cast<float*>(sm);   // the operands are consumed
        for (int ch = 0; ch < kTileN / 32; ++ch) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 32), v);
#pragma unroll
            for (int j = 0; j < 32; ++j) S[tid * 33 + j] = v[j];
            __syncthreads();
            float2 o[16];   // 16 independent loads, then the adds and stores
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int e = tid + u * 128, row = e >> 4, q = e & 15;
                const int i = i0 + row, c = c0 + ch * 16 + q;
                const bool ok_ = i < M && c < M && !(c >= J0 && c < J0 + nbo);
                o[u] = ok_ ? w[(long long)i * M + c] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int e = tid + u * 128, row = e >> 4, q = e & 15;
                const int i = i0 + row, c = c0 + ch * 16 + q;
                if (i >= M || c >= M || (c >= J0 && c < J0 + nbo)) continue;
                w[(long long)i * M + c] = make_float2(o[u].x + S[row * 33 + 2 * q], o[u].y + S[row * 33 + 2 * q + 1]);
            }
            __syncthreads();
        }
        // the next tile's operand writes must not overtake this tile's reads
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (!ok) {
        // the product did not signal in time: give it one more bounded wait
        // before the accumulator columns are released
        mbar_wait(bar, phase ^ 1u, err);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

// Launches the tensor-core update for the outer panel [J0, J0 + NO) of every
// slab (FP32 factors).
int lss3_update_tc(lss_ctx* c, float2* W, const float2* T64, int J0, int NO, cudaStream_t s) {
    Ctx3* d = c->d3;
    {
        std::lock_guard<std::mutex> lock(lss_config_mutex());
        long long& done = lss_dev_cache((const void*)f3_update_tc, 0);
        if (!done) {
            cudaError_t e = cudaFuncSetAttribute(f3_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
            if (e) return lss_check_cuda(c, e, "tensor-core update attribute");
            done = 1;
        }
    }
    const int tmax = (d->Mmax + 127) / 128;
    const long long slots = (long long)c->n_slabs * tmax * tmax;
    const int grid = (int)std::min<long long>(slots, 2LL * c->num_sms);
    f3_update_tc<<<grid, 128, kTcSmem, s>>>(d->d_slabs, c->n_slabs, W, T64, J0, NO, d->Mmax, tmax, c->d_err);
    return lss_check_cuda(c, cudaGetLastError(), "tensor-core update launch");
}

// The 3D mixed-precision factorization uses the tensor-core update unless
// LSS_TC_UPDATE=0 is set in the environment (the CUDA-core FP32 update with
// 16-column panels then runs; both reach the same factors to about 2e-6).
bool lss3_use_tc() {
    const char* v = std::getenv("LSS_TC_UPDATE");
    return !(v && v[0] == '0');
}
