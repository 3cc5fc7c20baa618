// Shared-memory Stockham line FFT used by the 2D and 3D LS operators.
#pragma once
#include "lss_common.cuh"

// Stockham FFT of one line of length L = 2^lg held in shared memory x; y is a
// second shared buffer.  Threads t = 0..nt-1 of the calling group cooperate;
// the whole block must call it together (it synchronises).  Returns the buffer
// that holds the result.  tw[k] = exp(-2 pi i k / L).
template <bool INV>
__device__ double2* fft_line(double2* x, double2* y, int L, int lg, const double2* __restrict__ tw,
                             int t, int nt) {
    int Ns = 1;
    if (lg & 1) {
        const int L2 = L >> 1;
        for (int j = t; j < L2; j += nt) {
            double2 a = x[j], c = x[j + L2];
            y[2 * j] = a + c;
            y[2 * j + 1] = a - c;
        }
        __syncthreads();
        double2* tmp = x; x = y; y = tmp;
        Ns = 2;
    }
    const int L4 = L >> 2;
    for (; Ns < L; Ns <<= 2) {
        const int st = L / (Ns << 2);
        for (int j = t; j < L4; j += nt) {
            const int q = j & (Ns - 1);
            double2 v0 = x[j], v1 = x[j + L4], v2 = x[j + 2 * L4], v3 = x[j + 3 * L4];
            if (Ns > 1) {
                double2 w1 = __ldg(&tw[q * st]), w2 = __ldg(&tw[2 * q * st]), w3 = __ldg(&tw[3 * q * st]);
                if (INV) { w1.y = -w1.y; w2.y = -w2.y; w3.y = -w3.y; }
                v1 = v1 * w1; v2 = v2 * w2; v3 = v3 * w3;
            }
            double2 a0 = v0 + v2, a1 = v0 - v2, a2 = v1 + v3, d = v1 - v3;
            double2 a3 = INV ? mk(-d.y, d.x) : mk(d.y, -d.x);
            const int o = ((j - q) << 2) + q;
            y[o] = a0 + a2;
            y[o + Ns] = a1 + a3;
            y[o + 2 * Ns] = a0 - a2;
            y[o + 3 * Ns] = a1 - a3;
        }
        __syncthreads();
        double2* tmp = x; x = y; y = tmp;
    }
    return x;
}
