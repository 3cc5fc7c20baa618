// Device helpers of the 3D path shared by the non-recursive and the recursive
// sweeps: PML profiles and classes, the 26-direction PML stencil (Eq. gamma in
// 3D) computed by one warp, the interior stencils, the medium lookup.
#pragma once
#include <cuda_runtime.h>

#include "lss_common.cuh"

namespace {

__device__ __forceinline__ double sigma_phys3(int q, int n, int b, double Cw) {
    if (q <= -1) { const double t = (q + 1.0) / b; return -Cw * t * t; }
    if (q >= n + 2) { const double t = (q - n - 2.0) / b; return Cw * t * t; }
    return 0.0;
}
__device__ __forceinline__ int pml_class3(int q, int n, int b) {
    if (q <= -1) return q + b + 1;
    if (q >= n + 2) return b + 1 + (q - n - 2);
    return 0;
}
__device__ __forceinline__ int class_index3(int cl, int n, int b) {
    if (cl == 0) return 0;
    if (cl <= b) return cl - b - 1;
    return n + 2 + (cl - b - 1);
}

constexpr int kGamWarps = 4;
struct GamSmem {
    double2 F[27][26];
    double2 E[3][3][3][2];   // [axis][d+1][scale][sign]
    double vn2[26];
    double2 q[27];
};

// One warp computes one stencil.  sig[axis][0..2] = sigma at offsets -1, 0, +1;
// w = local frequency.  F[o][r] = exp(i w r.(dp_o + i dsigma_o)) over the 26
// normalised directions r of {-1,0,1}^3 minus 0 (columns in lexicographic
// order); the exponential factors per axis, E(d, v) = exp(i w v (d h + i
// dsigma_d)) with v = +-1/sqrt(nnz(r)), and E(d, -v) has the conjugate phase
// and the reciprocal modulus of E(d, v).  The null vector of F^T is the last
// column of the unitary factor of a Householder QR of F (lane = column in the
// reflector updates).  out[o] = conj(gamma_o), unit norm, centre real positive;
// o = (d1+1)*9 + (d2+1)*3 + (d3+1).
__device__ void gamma3_warp(const double sig[3][3], double w, double h, GamSmem& S, double2* out) {
    const int lane = threadIdx.x & 31;
    if (lane < 27) {
        const int ax = lane / 9, d = (lane / 3) % 3 - 1, sc = lane % 3;
        const double v = sc == 0 ? 1.0 : (sc == 1 ? 0.70710678118654752440 : 0.57735026918962576451);
        const double re = d * h, im = sig[ax][d + 1] - sig[ax][1];
        double sn, cs;
        sincos(w * v * re, &sn, &cs);
        const double mag = exp(-w * v * im);
        S.E[ax][d + 1][sc][0] = mk(mag * cs, mag * sn);
        S.E[ax][d + 1][sc][1] = mk(cs / mag, -sn / mag);
    }
    __syncwarp();
    for (int e = lane; e < 27 * 26; e += 32) {
        const int o = e / 26, col = e % 26;
        const int rr = col < 13 ? col : col + 1;     // skip the zero direction
        const int r[3] = {rr / 9 - 1, (rr / 3) % 3 - 1, rr % 3 - 1};
        const int nnz = (r[0] != 0) + (r[1] != 0) + (r[2] != 0);
        const int dd[3] = {o / 9 - 1, (o / 3) % 3 - 1, o % 3 - 1};
        double2 f = mk(1.0, 0.0);
        for (int ax = 0; ax < 3; ++ax)
            if (r[ax] != 0) f = f * S.E[ax][dd[ax] + 1][nnz - 1][r[ax] < 0];
        S.F[o][col] = f;
    }
    __syncwarp();
    for (int k = 0; k < 26; ++k) {
        double2 x = lane >= k && lane < 27 ? S.F[lane][k] : mk(0.0, 0.0);
        double nx = cabs2(x);
        for (int o = 16; o > 0; o >>= 1) nx += __shfl_xor_sync(0xffffffffu, nx, o);
        nx = sqrt(nx);
        const double2 fkk = S.F[k][k];
        const double afk = sqrt(cabs2(fkk));
        const double2 ph = afk > 0 ? mk(fkk.x / afk, fkk.y / afk) : mk(1.0, 0.0);
        __syncwarp();
        if (lane == 0) S.F[k][k] = fkk - mk(-ph.x * nx, -ph.y * nx);   // v = x - alpha e_k
        __syncwarp();
        x = lane >= k && lane < 27 ? S.F[lane][k] : mk(0.0, 0.0);
        double v2 = cabs2(x);
        for (int o = 16; o > 0; o >>= 1) v2 += __shfl_xor_sync(0xffffffffu, v2, o);
        if (lane == 0) S.vn2[k] = v2;
        if (v2 > 0 && lane > k && lane < 26) {
            double2 dot = mk(0.0, 0.0);
            for (int i = k; i < 27; ++i) dot = cfma_conj(S.F[i][k], S.F[i][lane], dot);
            const double2 sd = (2.0 / v2) * dot;
            for (int i = k; i < 27; ++i) S.F[i][lane] = S.F[i][lane] - sd * S.F[i][k];
        }
        __syncwarp();
    }
    double2 q = lane == 26 ? mk(1.0, 0.0) : mk(0.0, 0.0);
    for (int k = 25; k >= 0; --k) {
        const double v2 = S.vn2[k];
        if (v2 == 0) continue;
        double2 t = lane >= k && lane < 27 ? S.F[lane][k] : mk(0.0, 0.0);
        double2 dot = lane >= k && lane < 27 ? mk(t.x * q.x + t.y * q.y, t.x * q.y - t.y * q.x) : mk(0.0, 0.0);
        for (int o = 16; o > 0; o >>= 1) {
            dot.x += __shfl_xor_sync(0xffffffffu, dot.x, o);
            dot.y += __shfl_xor_sync(0xffffffffu, dot.y, o);
        }
        if (lane >= k && lane < 27) q = q - ((2.0 / v2) * dot) * t;
    }
    double nq = lane < 27 ? cabs2(q) : 0.0;
    for (int o = 16; o > 0; o >>= 1) nq += __shfl_xor_sync(0xffffffffu, nq, o);
    nq = sqrt(nq);
    const double2 qc = mk(__shfl_sync(0xffffffffu, q.x, 13), __shfl_sync(0xffffffffu, q.y, 13));
    const double ac = sqrt(cabs2(qc));
    const double2 ph = mk(qc.x / ac, -qc.y / ac);
    if (lane < 27) {
        double2 g = (1.0 / nq) * (q * ph);
        if (lane == 13) g = mk(ac / nq, 0.0);
        out[lane] = conjc(g);
    }
    __syncwarp();
}

struct Stencil27 {
    double2 a_conj[27];
    double2 b_conj[27];
};

__device__ __forceinline__ double m3_at(const double* m, int n, int i1, int i2, int i3) {
    return (i1 >= 1 && i1 <= n && i2 >= 1 && i2 <= n && i3 >= 1 && i3 <= n)
               ? m[((size_t)(i1 - 1) * n + (i2 - 1)) * n + (i3 - 1)]
               : 0.0;
}

}  // namespace
