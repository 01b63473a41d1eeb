// fft.cuh -- power-of-two complex FFTs on data staged in shared memory.
//
// The oversampled grid of the NUFFT is transformed by two passes of 1-D FFTs (rows, then
// columns, and the reverse for the adjoint). Each CTA stages one row, or a block of adjacent
// columns, in shared memory; the 1-D transforms run there so that HBM sees one coalesced read
// and one coalesced write per pass.
#pragma once
#include "common.cuh"

namespace ivis {

__device__ __forceinline__ int bitrev(int n, int logL) {
    return (int)(__brev((unsigned)n) >> (32 - logL));
}

// In-place decimation-in-time radix-2 FFT of `ncols` independent columns of length L
// (L = 2^logL). Element n of column c must already sit at s[bitrev(n) * ncols + c]; on
// return output k of column c is at s[k * ncols + c]. SIGN = -1: sum x[n] e^{-2 pi i nk/L};
// SIGN = +1: sum x[n] e^{+2 pi i nk/L} (unnormalised). tw[j] = e^{-2 pi i j / L}, j < L/2.
// ncols must be a power of two. The caller synchronises before the call; the call ends
// with a __syncthreads.
template <typename C, int SIGN>
__device__ __forceinline__ void fft_dit_smem(C *s, int logL, int logc, const C *__restrict__ tw) {
    const int L = 1 << logL;
    const int ncols = 1 << logc;
    const int nbf = (L >> 1) << logc;
    for (int logh = 0; logh < logL; ++logh) {
        const int h = 1 << logh;
        for (int idx = threadIdx.x; idx < nbf; idx += blockDim.x) {
            const int c = idx & (ncols - 1);
            const int b = idx >> logc;
            const int j = b & (h - 1);
            const int i0 = ((b >> logh) << (logh + 1)) + j;
            const int i1 = i0 + h;
            C w = __ldg(&tw[j << (logL - 1 - logh)]);
            if (SIGN > 0) w.y = -w.y;
            C a = s[(i0 << logc) + c];
            C x = cmul(s[(i1 << logc) + c], w);
            s[(i0 << logc) + c] = a + x;
            s[(i1 << logc) + c] = a - x;
        }
        __syncthreads();
    }
}

}  // namespace ivis
