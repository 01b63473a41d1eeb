// fft.cuh -- power-of-two complex FFTs on lines staged in shared memory.
//
// The oversampled grid of the NUFFT is transformed by two passes of 1-D FFTs (rows, then
// columns, and the reverse for the adjoint). Each CTA stages a few rows, or a block of
// adjacent columns, in shared memory; HBM sees one coalesced read and one coalesced write per
// pass.
//
// Each line of length L = 2^logL is transformed by the Stockham auto-sort formulation
// (Govindaraju et al., "High performance discrete Fourier transforms on graphics
// processors", SC 2008): log_R(L) passes, in each of which a thread loads R elements spaced
// L/R apart, applies the pass twiddles, does a radix-R DFT in registers and stores the R
// results spaced Ns apart. Input and output are in natural order (no bit reversal). R = 16,
// with one final pass of radix 2, 4 or 8 when logL is not a multiple of 4. Shared-memory
// addresses are padded by one element every 16 (pidx) so the strided stores of the early
// passes do not pile onto one bank.
//
// The first pass's butterfly of thread j0 takes the line's elements j0 + r L/16 and the last
// pass's butterflies of that thread write exactly the elements j0 + m L/16. A kernel whose
// thread loads those elements itself (the packed passes: with an oversampling factor of 2,
// half of a forward line is zero padding and half of an adjoint line is dropped) can run the
// first pass from registers (first_pass_regs) and take the last pass's outputs in registers
// (last_pass_regs), skipping the staging round trip through shared memory at either end.
#pragma once
#include "common.cuh"

namespace ivis {

__host__ __device__ __forceinline__ int pidx(int e) { return e + (e >> 4); }

// Twiddle W_16^q = exp(-2 pi i q / 16) for q < 8 (cos and sin of q pi / 8).
__device__ __forceinline__ double cos16(int q) {
    constexpr double c[8] = {1.0, 0.92387953251128675613, 0.70710678118654752440,
                             0.38268343236508977173, 0.0, -0.38268343236508977173,
                             -0.70710678118654752440, -0.92387953251128675613};
    return c[q];
}
__device__ __forceinline__ double sin16(int q) {
    constexpr double s[8] = {0.0, 0.38268343236508977173, 0.70710678118654752440,
                             0.92387953251128675613, 1.0, 0.92387953251128675613,
                             0.70710678118654752440, 0.38268343236508977173};
    return s[q];
}

// In-register radix-2 decimation-in-frequency DFT of size R (natural-order input); output
// k ends up in v[bitrev_R(k)]. SIGN = -1 forward, +1 inverse (unnormalised).
template <typename C, int R, int SIGN>
__device__ __forceinline__ void dft_regs(C (&v)[R]) {
#pragma unroll
    for (int h = R / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int g = 0; g < R; g += 2 * h) {
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const C a = v[g + i], b = v[g + i + h];
                v[g + i] = a + b;
                C d = a - b;
                const int q = i * (16 / (2 * h));  // W_{2h}^i = W_16^q
                if (q != 0) {
                    if (q == 4) {  // multiply by -i (forward) or +i (inverse)
                        d = SIGN < 0 ? mk(d.y, -d.x) : mk(-d.y, d.x);
                    } else {
                        const auto c = (decltype(d.x))cos16(q);
                        const auto s = (decltype(d.x))(SIGN < 0 ? -sin16(q) : sin16(q));
                        d = mk(d.x * c - d.y * s, d.x * s + d.y * c);
                    }
                }
                v[g + i + h] = d;
            }
        }
    }
}

template <int R>
__device__ __forceinline__ constexpr int brev_c(int k) {
    int r = 0;
    for (int b = 1, o = R >> 1; b < R; b <<= 1, o >>= 1)
        if (k & b) r |= o;
    return r;
}

// One Stockham pass of radix RP on a line: element n at base[pidx(n * stride + off)].
// tpl threads (index j0 in [0, tpl)) each handle 16/RP butterfly groups.
template <typename C, int RP, int SIGN>
__device__ __forceinline__ void stockham_pass(C *base, int stride, int off, int L, int logL,
                                              int Ns, int logNs, int j0, int tpl,
                                              const C *__restrict__ tw) {
    constexpr int G = 16 / RP;
    C v[G][RP];
    const int LR = L / RP;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = j0 + g * tpl;
        const int k = j & (Ns - 1);
        // twiddle of input r: exp(SIGN 2 pi i k r / (Ns RP)), from this pass's block of the
        // table (adjacent k adjacent, so the lanes of a warp read one or two sectors)
        const int toff = 16 * (Ns - 1) / 15 + k;
#pragma unroll
        for (int r = 0; r < RP; ++r) {
            C x = base[pidx((j + r * LR) * stride + off)];
            if (r > 0 && k != 0) {
                C w = __ldg(&tw[toff + r * Ns]);
                if (SIGN > 0) w.y = -w.y;
                x = cmul(x, w);
            }
            v[g][r] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = j0 + g * tpl;
        C (&vv)[RP] = v[g];
        dft_regs<C, RP, SIGN>(vv);
        const int k = j & (Ns - 1);
        const int idxD = ((j >> logNs) << logNs) * RP + k;
#pragma unroll
        for (int r = 0; r < RP; ++r) base[pidx((idxD + r * Ns) * stride + off)] = vv[brev_c<RP>(r)];
    }
    __syncthreads();
}

// Full FFT of one line of length L = 2^logL (logL >= 4) held at base[pidx(n*stride + off)],
// by tpl = L/16 threads with line-local index j0. The caller synchronises before the call;
// the call ends synchronised. tw: the twiddles in pass order (built by fft_twiddles): for the pass
// with Ns = 2^logNs and radix R, tw[16 (Ns - 1) / 15 + r Ns + k] = exp(-2 pi i k r / (Ns R)),
// k < Ns, r < R (16 (Ns - 1) / 15 entries precede it: the earlier passes' 16 + 256 + ...).
template <typename C, int SIGN>
__device__ __forceinline__ void line_fft(C *base, int stride, int off, int logL, int j0,
                                         const C *__restrict__ tw) {
    const int L = 1 << logL;
    const int tpl = L >> 4;
    int logNs = 0;
    for (; logNs + 4 <= logL; logNs += 4)
        stockham_pass<C, 16, SIGN>(base, stride, off, L, logL, 1 << logNs, logNs, j0, tpl, tw);
    const int rem = logL - logNs;
    if (rem == 3) stockham_pass<C, 8, SIGN>(base, stride, off, L, logL, 1 << logNs, logNs, j0, tpl, tw);
    else if (rem == 2) stockham_pass<C, 4, SIGN>(base, stride, off, L, logL, 1 << logNs, logNs, j0, tpl, tw);
    else if (rem == 1) stockham_pass<C, 2, SIGN>(base, stride, off, L, logL, 1 << logNs, logNs, j0, tpl, tw);
}

// The first pass of line_fft (Ns = 1, radix 16) on an input held in registers: in[r] is the
// line's element j0 + r L/16, the inputs of this thread's butterfly. Writes the pass's output to
// the line; the caller synchronises before the next pass (line_fft_from with logNs0 = 4).
template <typename C, int SIGN>
__device__ __forceinline__ void first_pass_regs(C *base, int stride, int off, int j0, C (&in)[16]) {
    dft_regs<C, 16, SIGN>(in);
#pragma unroll
    for (int r = 0; r < 16; ++r) base[pidx((j0 * 16 + r) * stride + off)] = in[brev_c<16>(r)];
}

// The passes of line_fft from Ns = 2^logNs0 on (logNs0 a multiple of 4); with last_in_regs the
// final pass is left out (last_pass_regs runs it).
template <typename C, int SIGN>
__device__ __forceinline__ void line_fft_from(C *base, int stride, int off, int logL, int j0,
                                              const C *__restrict__ tw, int logNs0, bool last_in_regs) {
    const int L = 1 << logL;
    const int tpl = L >> 4;
    const int rem = logL & 3, n16 = logL >> 2;  // n16 radix-16 passes, then one of radix 2^rem
    const int n16_run = (rem == 0 && last_in_regs) ? n16 - 1 : n16;
    int logNs = logNs0;
    for (; logNs < 4 * n16_run; logNs += 4)
        stockham_pass<C, 16, SIGN>(base, stride, off, L, logL, 1 << logNs, logNs, j0, tpl, tw);
    if (rem == 0 || last_in_regs) return;
    if (rem == 3) stockham_pass<C, 8, SIGN>(base, stride, off, L, logL, 1 << logNs, logNs, j0, tpl, tw);
    else if (rem == 2) stockham_pass<C, 4, SIGN>(base, stride, off, L, logL, 1 << logNs, logNs, j0, tpl, tw);
    else stockham_pass<C, 2, SIGN>(base, stride, off, L, logL, 1 << logNs, logNs, j0, tpl, tw);
}

// The final pass (Ns = L / RP) of line_fft with its output handed to emit(m, value) as each
// butterfly finishes: m indexes the line's element j0 + m L/16 (the butterflies of this pass
// write exactly those elements, since each of the thread's G = 16 / RP groups j = j0 + g L/16
// has j < Ns). No shared-memory writes, so nothing to synchronise after it.
template <typename C, int RP, int SIGN, typename E>
__device__ __forceinline__ void last_pass_regs_rp(const C *base, int stride, int off, int L, int logNs, int j0,
                                                  const C *__restrict__ tw, E &&emit) {
    constexpr int G = 16 / RP;
    const int Ns = 1 << logNs, tpl = L >> 4, LR = L / RP;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = j0 + g * tpl;  // < Ns: k = j, output elements j + r Ns
        const int toff = 16 * (Ns - 1) / 15 + j;
        C v[RP];
#pragma unroll
        for (int r = 0; r < RP; ++r) {
            C x = base[pidx((j + r * LR) * stride + off)];
            if (r > 0 && j != 0) {
                C w = __ldg(&tw[toff + r * Ns]);
                if (SIGN > 0) w.y = -w.y;
                x = cmul(x, w);
            }
            v[r] = x;
        }
        dft_regs<C, RP, SIGN>(v);
#pragma unroll
        for (int r = 0; r < RP; ++r) emit(g + r * G, v[brev_c<RP>(r)]);  // element j0 + (g + r G) L/16
    }
}

template <typename C, int SIGN, typename E>
__device__ __forceinline__ void last_pass_regs(const C *base, int stride, int off, int logL, int j0,
                                               const C *__restrict__ tw, E &&emit) {
    const int L = 1 << logL;
    const int rem = logL & 3;
    const int logNs = rem == 0 ? logL - 4 : logL - rem;
    if (rem == 0) last_pass_regs_rp<C, 16, SIGN>(base, stride, off, L, logNs, j0, tw, emit);
    else if (rem == 3) last_pass_regs_rp<C, 8, SIGN>(base, stride, off, L, logNs, j0, tw, emit);
    else if (rem == 2) last_pass_regs_rp<C, 4, SIGN>(base, stride, off, L, logNs, j0, tw, emit);
    else last_pass_regs_rp<C, 2, SIGN>(base, stride, off, L, logNs, j0, tw, emit);
}

// Shared-memory elements needed for `lines` lines of length L (padded addressing).
__host__ __device__ inline int fft_smem_elems(int L, int lines) { return pidx(L * lines - 1) + 1; }

}  // namespace ivis
