// Overlap-add FFT filtering (include/filark.h, filark_fftfilt_*): the paper's
// benchmarked GPU filtering mode (Table 1, FFT-domain bandpass; Sec. 6.2,
// overlap-add chunked filtering), as a streaming operator with the chain's
// contract: y[n] = sum_{k<M} h[k] x[n-k], x before the stream start zero, the
// overlap tail carried across pushes.
//
// Each push is cut into blocks of at most L samples per channel.  A block b
// of len samples gives z = x_b * h (length len + M - 1) through an FFT of size
// N >= len + M - 1: Z = FFT(x_b) . H_N, z = IFFT(Z).  The outputs of the block
// are z[0, len) + tail[0, len); the tail becomes tail[len, ...) + z[len, ...).
// Two channels share one complex transform (x1 + i x2; h is real, so the real
// and imaginary parts of the result are the two convolutions).  N is the
// smallest size 2^k or 3 * 2^k that holds the block's convolution (a
// 1,500-sample push with 4,001 taps: 6144 rather than 8192), and H_N, the
// spectrum of the taps, is kept for every such size up to the largest.
//
// FFT: mixed-radix Stockham autosort in shared memory, one CTA per channel
// pair and block.  Passes: radix 3 first when 3 divides N, then one radix-2
// or radix-4 pass when log2 of the power-of-two part is not a multiple of 3,
// then radix 8; each thread does whole radix-R butterflies in registers.  The
// first forward pass reads the input block straight from global memory, the
// last forward pass multiplies by H_N, and the last inverse pass writes the
// outputs and the new tail straight to global memory.  The tail is
// double-buffered (read from one buffer, written to the other), so the
// epilogue needs no barrier.  Twiddles come from a host table made in double
// precision, one run of m values per pass (w_j = exp(-2 pi i j / (R m)),
// j < m, contiguous in j), staged in shared memory; a butterfly's powers
// w^2 .. w^7 are products of at most three table values' roundings.  Shared
// arrays are padded by one element per 16 (element i at i + i/16), which
// spreads the strided stores of the early passes over the banks.
// N <= 8192; up to 6144 two CTAs of N / 16 threads share an SM.
//
// Filters longer than 4096 taps whose block would not fit the 8192-point
// transform use a partitioned convolution: the taps are cut into P partitions
// of B = 4096 (the last shorter), h_p = h[pB, pB + B), with one spectrum per
// partition and transform size; a block of len <= B samples is transformed
// once (its spectrum X stays in shared memory) and each partition adds
// IFFT(X H_p), the block convolved with h_p, at block position pB.  The
// partitions run in order inside the CTA: positions [pB, (p+1)B) are owned by
// partition p (it adds the old tail there), and p's overhang past (p+1)B
// (len - 1 positions) goes to the new tail as a partial sum that p + 1
// completes.  Outputs are positions < len, which only partition 0 reaches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "filark_internal.h"
#include "host_trace.h"

using namespace filark;

namespace {

constexpr int kFftMaxThreads = 1024;
constexpr int kFftMaxN = 8192;
constexpr int kMaxPass = 6;
constexpr size_t kTwoCtaSmem = 110 * 1024;   // at most this much shared memory: two CTAs per SM

// padded shared-memory position of element i
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
int pad_h(int i) { return i + (i >> 4); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// z * (d i), d = -1 forward, +1 inverse
template <bool INV>
__device__ __forceinline__ float2 rot(float2 z) {
    return INV ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
}

// In-register DFT of size R: y_q = sum_r x_r exp(d 2 pi i r q / R).
template <bool INV>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
    const float2 s0 = cadd(a0, a2), s1 = csub(a0, a2), s2 = cadd(a1, a3), s3 = rot<INV>(csub(a1, a3));
    a0 = cadd(s0, s2);
    a2 = csub(s0, s2);
    a1 = cadd(s1, s3);
    a3 = csub(s1, s3);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&x)[R]) {
    if constexpr (R == 2) {
        const float2 u = x[0];
        x[0] = cadd(u, x[1]);
        x[1] = csub(u, x[1]);
    } else if constexpr (R == 3) {
        // y0 = x0 + (x1 + x2), y1,2 = x0 - (x1 + x2)/2 +- d i (sqrt(3)/2)(x1 - x2)
        const float h = 0.86602540378443865f;
        const float2 s = cadd(x[1], x[2]);
        const float2 t = make_float2(x[0].x - 0.5f * s.x, x[0].y - 0.5f * s.y);
        const float2 u = rot<INV>(csub(x[1], x[2]));
        x[0] = cadd(x[0], s);
        x[1] = make_float2(t.x + h * u.x, t.y + h * u.y);
        x[2] = make_float2(t.x - h * u.x, t.y - h * u.y);
    } else if constexpr (R == 4) {
        dft4<INV>(x[0], x[1], x[2], x[3]);
    } else {
        // even / odd halves, then y_q = E_q + w8^q O_q, y_{q+4} = E_q - w8^q O_q
        dft4<INV>(x[0], x[2], x[4], x[6]);
        dft4<INV>(x[1], x[3], x[5], x[7]);
        const float c = 0.70710678118654752f;
        const float d = INV ? 1.f : -1.f;
        const float2 o1 = make_float2(c * (x[3].x - d * x[3].y), c * (x[3].y + d * x[3].x));
        const float2 o2 = rot<INV>(x[5]);
        const float2 o3 = make_float2(c * (-x[7].x - d * x[7].y), c * (-x[7].y + d * x[7].x));
        const float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6], o0 = x[1];
        x[0] = cadd(e0, o0);
        x[4] = csub(e0, o0);
        x[1] = cadd(e1, o1);
        x[5] = csub(e1, o1);
        x[2] = cadd(e2, o2);
        x[6] = csub(e2, o2);
        x[3] = cadd(e3, o3);
        x[7] = csub(e3, o3);
    }
}

// x_r *= w^r (w conjugated for the inverse)
template <int R, bool INV>
__device__ __forceinline__ void twiddle(float2 (&x)[R], float2 w) {
    if (INV) w.y = -w.y;
    if constexpr (R == 2) {
        x[1] = cmul(x[1], w);
    } else if constexpr (R == 3) {
        x[1] = cmul(x[1], w);
        x[2] = cmul(x[2], cmul(w, w));
    } else if constexpr (R == 4) {
        const float2 w2 = cmul(w, w);
        x[1] = cmul(x[1], w);
        x[2] = cmul(x[2], w2);
        x[3] = cmul(x[3], cmul(w2, w));
    } else {
        const float2 w2 = cmul(w, w), w4 = cmul(w2, w2), w3 = cmul(w2, w);
        x[1] = cmul(x[1], w);
        x[2] = cmul(x[2], w2);
        x[3] = cmul(x[3], w3);
        x[4] = cmul(x[4], w4);
        x[5] = cmul(x[5], cmul(w4, w));
        x[6] = cmul(x[6], cmul(w4, w2));
        x[7] = cmul(x[7], cmul(w4, w3));
    }
}

// One transform size: its passes (radix R[p] combining sub-transforms of
// length m[p]; twiddle run at toff[p]).
struct FftParams {
    int N, M;
    int npass;
    int R[kMaxPass], m[kMaxPass], toff[kMaxPass];
    unsigned mdiv[kMaxPass];   // ceil(2^32 / m): t / m = umulhi(t, mdiv) for t, m < 2^16 (m > 1)
    int twlen;          // entries of the per-pass twiddle table
    float scale;        // 1 / N
};

// Where a pass reads from and writes to.
enum { SRC_SMEM = 0, SRC_GIN = 1, SRC_SMEM_H = 2 };
enum { DST_SMEM = 0, DST_SMEM_H = 1, DST_GOUT = 2, DST_GOUT_PART = 3 };

struct BlockIO {
    const float *x;         // input block, time-major, row stride ldx
    long long ldx;
    int len;                // samples in this block
    int c1;                 // first channel of the pair (c1 + 1 the second, if has2)
    bool has2;
    bool pair_in, pair_out; // both channels as one 8-byte access (even ld, 8-byte aligned rows)
    const float2 *H;        // [N] spectrum of the taps
    const float *told;      // [C][M-1] tail before this block (NULL if M = 1)
    float *tnew;            // [C][M-1] tail after this block
    float *y;               // output block, row stride ldy
    long long ldy;
    int T1;                 // M - 1
    float scale;
    // partitioned convolution (M + block length - 1 above the largest FFT):
    // this transform is the block convolved with taps [off, off + lenp) of
    // partition `part`; partitions are B taps long (the last may be shorter)
    int off, lenp, B, part;
    bool last_part;
};

// One Stockham pass of radix R: sub-transforms of length m are combined R at
// a time.  Butterfly t (< N/R) reads elements t + r N/R, scales them by w^r
// with w = exp(d 2 pi i j / (R m)) = tw[j] (this pass's run of the table),
// j = t mod m, and writes the radix-R DFT to (t - j) R + j + q m.
template <int R, bool INV, int SRC, int DST>
__device__ __forceinline__ void radix_pass(const float2 *__restrict__ a, float2 *__restrict__ b, int N, int m,
                                           unsigned mdiv, const float2 *tw, const BlockIO &io) {
    const int stride = N / R;
    for (int t = threadIdx.x; t < stride; t += blockDim.x) {
        const int k = m == 1 ? t : (int)__umulhi((unsigned)t, mdiv), j = t - k * m;
        const int base = k * R * m + j;
        // the old tail values this butterfly's outputs add (issued first: they
        // do not depend on the transform)
        float2 told_q[DST == DST_GOUT || DST == DST_GOUT_PART ? R : 1];
        if constexpr (DST == DST_GOUT) {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = base + q * m;
                told_q[q] = make_float2(0.f, 0.f);
                if (i < io.T1) {
                    told_q[q].x = __ldg(io.told + (long long)io.c1 * io.T1 + i);
                    if (io.has2) told_q[q].y = __ldg(io.told + (long long)(io.c1 + 1) * io.T1 + i);
                }
            }
        } else if constexpr (DST == DST_GOUT_PART) {
            // what block position j = off + i already holds: the old tail,
            // added by the partition that owns j (j in [part B, (part + 1) B),
            // or the last partition), and the previous partition's overhang
            // into [part B, part B + len - 1), which it left in the new tail
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = base + q * m, j = io.off + i;
                told_q[q] = make_float2(0.f, 0.f);
                if (i < io.len + io.lenp - 1) {
                    if ((i < io.B || io.last_part) && j < io.T1) {
                        told_q[q].x = __ldg(io.told + (long long)io.c1 * io.T1 + j);
                        if (io.has2) told_q[q].y = __ldg(io.told + (long long)(io.c1 + 1) * io.T1 + j);
                    }
                    if (io.part > 0 && i < io.len - 1) {
                        // written by this CTA in the previous partition (plain loads)
                        told_q[q].x += io.tnew[(long long)io.c1 * io.T1 + (j - io.len)];
                        if (io.has2) told_q[q].y += io.tnew[(long long)(io.c1 + 1) * io.T1 + (j - io.len)];
                    }
                }
            }
        }
        float2 x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = t + r * stride;
            if constexpr (SRC == SRC_GIN) {
                float re = 0.f, im = 0.f;
                if (i < io.len) {
                    const float *src = io.x + (long long)i * io.ldx + io.c1;
                    if (io.pair_in) {
                        const float2 v = __ldg(reinterpret_cast<const float2 *>(src));
                        re = v.x;
                        im = v.y;
                    } else {
                        re = __ldg(src);
                        if (io.has2) im = __ldg(src + 1);
                    }
                }
                x[r] = make_float2(re, im);
            } else if constexpr (SRC == SRC_SMEM_H) {
                x[r] = cmul(a[pad(i)], __ldg(io.H + i));
            } else {
                x[r] = a[pad(i)];
            }
        }
        if (m > 1) twiddle<R, INV>(x, tw[j]);
        dft<R, INV>(x);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = base + q * m;
            if constexpr (DST == DST_SMEM) {
                b[pad(i)] = x[q];
            } else if constexpr (DST == DST_SMEM_H) {
                b[pad(i)] = cmul(x[q], __ldg(io.H + i));
            } else if constexpr (DST == DST_GOUT_PART) {
                // block position j = off + i: an output (j < len, partition 0
                // only, as B >= len) or new tail entry j - len
                if (i < io.len + io.lenp - 1) {
                    const int j = io.off + i;
                    const float v1 = x[q].x * io.scale + told_q[q].x, v2 = x[q].y * io.scale + told_q[q].y;
                    if (j < io.len) {
                        float *dst = io.y + (long long)j * io.ldy + io.c1;
                        if (io.pair_out) {
                            *reinterpret_cast<float2 *>(dst) = make_float2(v1, v2);
                        } else {
                            dst[0] = v1;
                            if (io.has2) dst[1] = v2;
                        }
                    } else {
                        io.tnew[(long long)io.c1 * io.T1 + (j - io.len)] = v1;
                        if (io.has2) io.tnew[(long long)(io.c1 + 1) * io.T1 + (j - io.len)] = v2;
                    }
                }
            } else {
                // z[i] (scaled) plus the old tail gives output i (i < len) or
                // new tail entry i - len (len <= i < len + M - 1)
                if (i < io.len + io.T1) {
                    const float v1 = x[q].x * io.scale + told_q[q].x, v2 = x[q].y * io.scale + told_q[q].y;
                    if (i < io.len) {
                        float *dst = io.y + (long long)i * io.ldy + io.c1;
                        if (io.pair_out) {
                            *reinterpret_cast<float2 *>(dst) = make_float2(v1, v2);
                        } else {
                            dst[0] = v1;
                            if (io.has2) dst[1] = v2;
                        }
                    } else {
                        io.tnew[(long long)io.c1 * io.T1 + (i - io.len)] = v1;
                        if (io.has2) io.tnew[(long long)(io.c1 + 1) * io.T1 + (i - io.len)] = v2;
                    }
                }
            }
        }
    }
}

template <bool INV, int SRC, int DST>
__device__ __forceinline__ void radix_pass_any(int R, const float2 *a, float2 *b, int N, int m, unsigned mdiv,
                                               const float2 *tw, const BlockIO &io) {
    switch (R) {
    case 2: radix_pass<2, INV, SRC, DST>(a, b, N, m, mdiv, tw, io); break;
    case 3: radix_pass<3, INV, SRC, DST>(a, b, N, m, mdiv, tw, io); break;
    case 4: radix_pass<4, INV, SRC, DST>(a, b, N, m, mdiv, tw, io); break;
    default: radix_pass<8, INV, SRC, DST>(a, b, N, m, mdiv, tw, io); break;
    }
}

// Forward transform of the input block (read from global memory), times H
// when io.H is set; the result is left in the returned buffer.
__device__ float2 *fft_forward(const FftParams &fp, float2 *a, float2 *b, const float2 *tw, const BlockIO &io) {
    for (int p = 0; p < fp.npass; ++p) {
        const bool last = p == fp.npass - 1;
        const float2 *twp = tw + fp.toff[p];
        const int R = fp.R[p], m = fp.m[p];
        const unsigned md = fp.mdiv[p];
        if (p == 0) {
            if (last && io.H) radix_pass_any<false, SRC_GIN, DST_SMEM_H>(R, a, b, fp.N, m, md, twp, io);
            else radix_pass_any<false, SRC_GIN, DST_SMEM>(R, a, b, fp.N, m, md, twp, io);
        } else {
            if (last && io.H) radix_pass_any<false, SRC_SMEM, DST_SMEM_H>(R, a, b, fp.N, m, md, twp, io);
            else radix_pass_any<false, SRC_SMEM, DST_SMEM>(R, a, b, fp.N, m, md, twp, io);
        }
        __syncthreads();
        float2 *tmp = a;
        a = b;
        b = tmp;
    }
    return a;
}

// Inverse transform of a (unscaled); the last pass writes outputs and tail.
__device__ void fft_inverse_out(const FftParams &fp, float2 *a, float2 *b, const float2 *tw, const BlockIO &io) {
    for (int p = 0; p < fp.npass; ++p) {
        const float2 *twp = tw + fp.toff[p];
        if (p == fp.npass - 1) {
            radix_pass_any<true, SRC_SMEM, DST_GOUT>(fp.R[p], a, b, fp.N, fp.m[p], fp.mdiv[p], twp, io);
        } else {
            radix_pass_any<true, SRC_SMEM, DST_SMEM>(fp.R[p], a, b, fp.N, fp.m[p], fp.mdiv[p], twp, io);
            __syncthreads();
            float2 *tmp = a;
            a = b;
            b = tmp;
        }
    }
}

// Inverse transform of X times io.H (the first pass multiplies as it reads, so
// X is kept for the next partition), through the work buffers w1 and w2; the
// last pass adds this partition's convolution into the outputs and the new
// tail.  Needs at least two passes.
__device__ void fft_inverse_part(const FftParams &fp, const float2 *X, float2 *w1, float2 *w2, const float2 *tw,
                                 const BlockIO &io) {
    const float2 *a = X;
    float2 *b = w1;
    for (int p = 0; p < fp.npass; ++p) {
        const float2 *twp = tw + fp.toff[p];
        if (p == fp.npass - 1) {
            radix_pass_any<true, SRC_SMEM, DST_GOUT_PART>(fp.R[p], a, b, fp.N, fp.m[p], fp.mdiv[p], twp, io);
        } else {
            if (p == 0) radix_pass_any<true, SRC_SMEM_H, DST_SMEM>(fp.R[p], a, b, fp.N, fp.m[p], fp.mdiv[p], twp, io);
            else radix_pass_any<true, SRC_SMEM, DST_SMEM>(fp.R[p], a, b, fp.N, fp.m[p], fp.mdiv[p], twp, io);
            __syncthreads();
            a = b;
            b = (b == w1) ? w2 : w1;
        }
    }
}

// One CTA per (channel pair, block) of a launch; the blocks of one launch are
// consecutive and independent given the tail, so a launch covers exactly one
// block per channel pair and the host launches the blocks of a push in order.
__global__ void __launch_bounds__(kFftMaxThreads) fftfilt_block_kernel(const __grid_constant__ FftParams fp,
                                                                       const float *__restrict__ x, long long ldx,
                                                                       int len, int C,
                                                                       const float2 *__restrict__ H,
                                                                       const float2 *__restrict__ tw,
                                                                       const float *__restrict__ told,
                                                                       float *__restrict__ tnew,
                                                                       float *__restrict__ y, long long ldy) {
    extern __shared__ float2 sm[];
    const int NP = pad(fp.N);
    float2 *stw = sm + 2 * NP;
    for (int i = threadIdx.x; i < fp.twlen; i += blockDim.x) stw[i] = __ldg(tw + i);
    {
        // start the old tail of both channels (contiguous) on its way to L2
        const int T1 = fp.M - 1, c1 = 2 * blockIdx.x;
        const long long n = (long long)T1 * min(2, C - c1);
        const long long off = (long long)threadIdx.x * 32;   // one 128-byte line per thread
        for (long long e = off; e < n; e += (long long)blockDim.x * 32)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(told + (long long)c1 * T1 + e));
    }
    BlockIO io;
    io.x = x;
    io.ldx = ldx;
    io.len = len;
    io.c1 = 2 * blockIdx.x;
    io.has2 = io.c1 + 1 < C;
    // c1 is even: with an even row stride and 8-byte aligned bases the pair is one float2
    io.pair_in = io.has2 && (ldx & 1) == 0 && ((uintptr_t)x & 7u) == 0;
    io.pair_out = io.has2 && (ldy & 1) == 0 && ((uintptr_t)y & 7u) == 0;
    io.H = H;
    io.told = told;
    io.tnew = tnew;
    io.y = y;
    io.ldy = ldy;
    io.T1 = fp.M - 1;
    io.scale = fp.scale;
    __syncthreads();
    float2 *X = fft_forward(fp, sm, sm + NP, stw, io);
    fft_inverse_out(fp, X, X == sm ? sm + NP : sm, stw, io);
}

// Partitioned convolution of one (channel pair, block): the block's spectrum X
// stays in shared memory and each partition p of the taps adds X H_p, inverse
// transformed, at block position p B; partitions run in order, so the
// overhang of partition p into the next one (len - 1 positions) is left in
// the new tail and completed by p + 1.  Three padded buffers.
__global__ void __launch_bounds__(kFftMaxThreads) fftfilt_part_kernel(const __grid_constant__ FftParams fp,
                                                                      const float *__restrict__ x, long long ldx,
                                                                      int len, int C, int n_parts, int B,
                                                                      const float2 *__restrict__ Hparts,
                                                                      const float2 *__restrict__ tw,
                                                                      const float *__restrict__ told,
                                                                      float *__restrict__ tnew,
                                                                      float *__restrict__ y, long long ldy) {
    extern __shared__ float2 sm[];
    const int NP = pad(fp.N);
    float2 *stw = sm + 3 * NP;
    for (int i = threadIdx.x; i < fp.twlen; i += blockDim.x) stw[i] = __ldg(tw + i);
    BlockIO io;
    io.x = x;
    io.ldx = ldx;
    io.len = len;
    io.c1 = 2 * blockIdx.x;
    io.has2 = io.c1 + 1 < C;
    io.pair_in = io.has2 && (ldx & 1) == 0 && ((uintptr_t)x & 7u) == 0;
    io.pair_out = io.has2 && (ldy & 1) == 0 && ((uintptr_t)y & 7u) == 0;
    io.H = nullptr;
    io.told = told;
    io.tnew = tnew;
    io.y = y;
    io.ldy = ldy;
    io.T1 = fp.M - 1;
    io.scale = fp.scale;
    io.B = B;
    __syncthreads();
    const float2 *X = fft_forward(fp, sm, sm + NP, stw, io);
    float2 *w1 = X == sm ? sm + NP : sm, *w2 = sm + 2 * NP;
    for (int part = 0; part < n_parts; ++part) {
        io.H = Hparts + (long long)part * fp.N;
        io.part = part;
        io.off = part * B;
        io.lenp = min(B, fp.M - part * B);
        io.last_part = part == n_parts - 1;
        fft_inverse_part(fp, X, w1, w2, stw, io);
        // the next partition reads this one's overhang from the new tail and
        // reuses the work buffers
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kFftMaxThreads) fft_of_taps_kernel(const __grid_constant__ FftParams fp,
                                                                     const float *__restrict__ h, int n,
                                                                     const float2 *__restrict__ tw,
                                                                     float2 *__restrict__ H) {
    extern __shared__ float2 sm[];
    const int NP = pad(fp.N);
    float2 *stw = sm + 2 * NP;
    for (int i = threadIdx.x; i < fp.twlen; i += blockDim.x) stw[i] = __ldg(tw + i);
    __syncthreads();
    BlockIO io{};
    io.x = h;
    io.ldx = 1;
    io.len = n;
    io.c1 = 0;
    io.has2 = false;
    io.H = nullptr;
    const float2 *r = fft_forward(fp, sm, sm + NP, stw, io);
    for (int i = threadIdx.x; i < fp.N; i += blockDim.x) H[i] = r[pad(i)];
}

// two padded buffers and the twiddle table (three for the partitioned kernel)
size_t fft_smem(int N, int twlen, int buffers = 2) {
    return sizeof(float2) * ((size_t)buffers * (size_t)pad_h(N) + (size_t)twlen);
}

// sizes 2^k and 3 * 2^k, 2 <= N <= kFftMaxN
bool fft_size_ok(int N) {
    if (N < 2 || N > kFftMaxN) return false;
    const int p = N % 3 == 0 ? N / 3 : N;
    return (p & (p - 1)) == 0;
}

// smallest such size >= n (0 if none)
int fft_size_at_least(int n) {
    for (int N = std::max(n, 2); N <= kFftMaxN; ++N)
        if (fft_size_ok(N)) return N;
    return 0;
}

// Passes, twiddle runs and launch shape of one size.
struct FftSize {
    FftParams fp{};
    std::vector<float2> tw;
    int threads = 0;
    size_t smem = 0;
    float2 *d_H = nullptr, *d_tw = nullptr;
};

void make_size(int N, int M, FftSize &z, int buffers) {
    FftParams &fp = z.fp;
    std::memset(&fp, 0, sizeof(fp));
    fp.N = N;
    fp.M = M;
    fp.scale = 1.0f / (float)N;
    int rest = N;
    std::vector<int> radices;
    if (rest % 3 == 0) {
        radices.push_back(3);
        rest /= 3;
    }
    int a = 0;
    while ((1 << a) < rest) ++a;
    if (a % 3) radices.push_back(1 << (a % 3));
    for (int i = 0; i < a / 3; ++i) radices.push_back(8);
    fp.npass = (int)radices.size();
    int m = 1;
    z.tw.clear();
    for (int p = 0; p < fp.npass; ++p) {
        fp.R[p] = radices[(size_t)p];
        fp.m[p] = m;
        fp.mdiv[p] = m > 1 ? (unsigned)((((uint64_t)1 << 32) + (uint64_t)m - 1) / (uint64_t)m) : 0u;
        fp.toff[p] = (int)z.tw.size();
        if (m > 1) {
            const int Rm = m * fp.R[p];
            for (int j = 0; j < m; ++j) {
                const double ang = -2.0 * 3.14159265358979323846 * (double)j / (double)Rm;
                z.tw.push_back(make_float2((float)std::cos(ang), (float)std::sin(ang)));
            }
        }
        m *= fp.R[p];
    }
    if (z.tw.empty()) z.tw.push_back(make_float2(1.f, 0.f));
    fp.twlen = (int)z.tw.size();
    z.smem = fft_smem(N, fp.twlen, buffers);
    // two CTAs of N / 16 threads per SM where their shared memory fits, else
    // one CTA of up to N / 8 threads
    z.threads = z.smem <= kTwoCtaSmem ? std::max(32, N / 16) : std::max(32, std::min(kFftMaxThreads, N / 8));
}

// Partition length of the partitioned mode: blocks of at most this many
// samples and partitions of this many taps fit the largest transform.
constexpr int kPartB = kFftMaxN / 2;
constexpr int kMaxTaps = 1 << 24;

}  // namespace

struct filark_fftfilt {
    int device = 0, C = 0, M = 0, L = 0, Nmax = 0;
    int P = 0;                      // partitions of kPartB taps (0: one transform holds block + taps)
    long long max_chunk = 0;
    std::vector<FftSize> sizes;     // ascending N: every size from the first >= M (or >= kPartB) up to Nmax;
                                    // d_H holds P spectra of N points each in the partitioned mode
    float *tail[2] = {nullptr, nullptr};   // [C][M-1] each; tail[cur] is current
    int cur = 0;
};

namespace {

void free_fftfilt(filark_fftfilt *f) {
    for (FftSize &z : f->sizes) {
        if (z.d_H) cudaFree(z.d_H);
        if (z.d_tw) cudaFree(z.d_tw);
    }
    if (f->tail[0]) cudaFree(f->tail[0]);
    if (f->tail[1]) cudaFree(f->tail[1]);
    delete f;
}

}  // namespace

extern "C" {

filark_status filark_fftfilt_create(int n_channels, int n_taps, const double *taps, int block_len,
                                    int64_t max_chunk, int cuda_device, filark_fftfilt **out) {
    if (!out) return fail_with(FILARK_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_channels < 1 || n_taps < 1 || !taps || max_chunk < 1)
        return fail_with(FILARK_EINVAL, "need n_channels >= 1, n_taps >= 1, taps, max_chunk >= 1");
    for (int k = 0; k < n_taps; ++k)
        if (!std::isfinite(taps[k])) return fail_with(FILARK_EINVAL, "non-finite tap");
    if (n_taps > kMaxTaps) return fail_with(FILARK_EINVAL, "n_taps above 2^24");
    long long L = block_len;
    if (L <= 0) {
        // default: the largest block with N = 2 next_pow2(M) or more
        long long n = 1;
        while (n < 2LL * n_taps) n <<= 1;
        L = n - n_taps + 1;
    }
    // Block and taps above the largest transform: up to kPartB taps the block
    // is shortened to fit (at least kFftMaxN - kPartB + 1 samples); longer
    // filters use the partitioned convolution, partitions of kPartB taps and
    // blocks of at most kPartB samples.
    const bool parted = L + n_taps - 1 > kFftMaxN && n_taps > kPartB;
    if (parted) L = std::min<long long>(block_len > 0 ? block_len : kPartB, kPartB);
    else if (L + n_taps - 1 > kFftMaxN) L = kFftMaxN - n_taps + 1;
    filark_fftfilt *f = new (std::nothrow) filark_fftfilt();
    if (!f) return fail_with(FILARK_ENOMEM, "host allocation failed");
    f->device = cuda_device;
    f->C = n_channels;
    f->M = n_taps;
    f->L = (int)L;
    f->max_chunk = max_chunk;
    f->P = parted ? (n_taps + kPartB - 1) / kPartB : 0;
    const int span = parted ? kPartB : n_taps;   // taps one transform convolves with
    f->Nmax = fft_size_at_least((int)L + span - 1);
    for (int N = fft_size_at_least(span); N > 0 && N <= f->Nmax; N = fft_size_at_least(N + 1)) {
        f->sizes.emplace_back();
        make_size(N, n_taps, f->sizes.back(), parted ? 3 : 2);
    }
    DeviceGuard dg(cuda_device);
    if (!dg.ok) {
        delete f;
        return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    }
    std::vector<float> hf((size_t)n_taps);
    for (int k = 0; k < n_taps; ++k) hf[(size_t)k] = (float)taps[k];
    float *dh = nullptr;
    cudaError_t e = cudaMalloc(&dh, sizeof(float) * (size_t)n_taps);
    if (e == cudaSuccess) e = cudaMemcpy(dh, hf.data(), sizeof(float) * hf.size(), cudaMemcpyHostToDevice);
    const size_t tail_bytes = sizeof(float) * (size_t)n_channels * (size_t)(n_taps - 1);
    if (e == cudaSuccess && n_taps > 1) e = cudaMalloc(&f->tail[0], tail_bytes);
    if (e == cudaSuccess && n_taps > 1) e = cudaMalloc(&f->tail[1], tail_bytes);
    size_t max_smem = 0;
    for (const FftSize &z : f->sizes) max_smem = std::max(max_smem, z.smem);
    if (e == cudaSuccess)
        e = parted ? cudaFuncSetAttribute(fftfilt_part_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)max_smem)
                   : cudaFuncSetAttribute(fftfilt_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)max_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft_of_taps_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
    const int n_spec = parted ? f->P : 1;
    for (FftSize &z : f->sizes) {
        if (e == cudaSuccess) e = cudaMalloc(&z.d_H, sizeof(float2) * (size_t)z.fp.N * (size_t)n_spec);
        if (e == cudaSuccess) e = cudaMalloc(&z.d_tw, sizeof(float2) * z.tw.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(z.d_tw, z.tw.data(), sizeof(float2) * z.tw.size(), cudaMemcpyHostToDevice);
        // the spectrum of the taps, or of each partition of kPartB taps
        for (int q = 0; q < n_spec && e == cudaSuccess; ++q) {
            const int n = parted ? std::min(kPartB, n_taps - q * kPartB) : n_taps;
            fft_of_taps_kernel<<<1, z.threads, z.smem>>>(z.fp, dh + (size_t)q * kPartB, n, z.d_tw,
                                                        z.d_H + (size_t)q * z.fp.N);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && f->tail[0]) e = cudaMemset(f->tail[0], 0, tail_bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (dh) cudaFree(dh);
    if (e != cudaSuccess) {
        free_fftfilt(f);
        return fail_cuda_with(e, "fftfilt create");
    }
    *out = f;
    return FILARK_OK;
}

filark_status filark_fftfilt_push(filark_fftfilt *f, const float *d_in, int64_t ld_in, int64_t n_samples,
                                  float *d_out, int64_t ld_out, filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_fftfilt_push");
    if (!f) return fail_with(FILARK_EINVAL, "filter is NULL");
    if (n_samples < 0 || n_samples > f->max_chunk) return fail_with(FILARK_EINVAL, "n_samples must be in [0, max_chunk]");
    if (n_samples == 0) return FILARK_OK;
    if (!d_in || !d_out || ld_in < f->C || ld_out < f->C) return fail_with(FILARK_EINVAL, "buffers NULL or ld < C");
    const size_t in_bytes = sizeof(float) * (size_t)((n_samples - 1) * ld_in + f->C);
    const size_t out_bytes = sizeof(float) * (size_t)((n_samples - 1) * ld_out + f->C);
    const char *pi = (const char *)d_in, *po = (const char *)d_out;
    if (pi < po + out_bytes && po < pi + in_bytes) return fail_with(FILARK_EINVAL, "output overlaps the input");
    DeviceGuard dg(f->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned pairs = (unsigned)((f->C + 1) / 2);
    for (int64_t t = 0; t < n_samples; t += f->L) {
        const int len = (int)std::min<int64_t>(f->L, n_samples - t);
        // the smallest size that holds this block's convolution (with the
        // taps, or with one partition of them)
        const int span = f->P ? kPartB : f->M;
        const FftSize *z = &f->sizes.back();
        for (const FftSize &c : f->sizes)
            if (c.fp.N >= len + span - 1) {
                z = &c;
                break;
            }
        if (f->P)
            fftfilt_part_kernel<<<pairs, z->threads, z->smem, s>>>(z->fp, d_in + t * ld_in, ld_in, len, f->C, f->P,
                                                                     kPartB, z->d_H, z->d_tw, f->tail[f->cur],
                                                                     f->tail[1 - f->cur], d_out + t * ld_out, ld_out);
        else
            fftfilt_block_kernel<<<pairs, z->threads, z->smem, s>>>(z->fp, d_in + t * ld_in, ld_in, len, f->C,
                                                                      z->d_H, z->d_tw, f->tail[f->cur],
                                                                      f->tail[1 - f->cur], d_out + t * ld_out, ld_out);
        f->cur = 1 - f->cur;
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FILARK_OK : fail_cuda_with(e, "fftfilt push");
}

filark_status filark_fftfilt_reset(filark_fftfilt *f, filark_stream_t stream) {
    if (!f) return fail_with(FILARK_EINVAL, "filter is NULL");
    DeviceGuard dg(f->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    if (!f->tail[0]) return FILARK_OK;
    const cudaError_t e = cudaMemsetAsync(f->tail[f->cur], 0, sizeof(float) * (size_t)f->C * (f->M - 1),
                                          (cudaStream_t)stream);
    return e == cudaSuccess ? FILARK_OK : fail_cuda_with(e, "fftfilt reset");
}

filark_status filark_fftfilt_get_info(const filark_fftfilt *f, int *fft_len, int *block_len) {
    if (!f) return fail_with(FILARK_EINVAL, "filter is NULL");
    if (fft_len) *fft_len = f->Nmax;
    if (block_len) *block_len = f->L;
    return FILARK_OK;
}

filark_status filark_fftfilt_destroy(filark_fftfilt *f) {
    if (!f) return FILARK_OK;
    DeviceGuard dg(f->device);
    cudaDeviceSynchronize();
    free_fftfilt(f);
    return FILARK_OK;
}

}  // extern "C"
