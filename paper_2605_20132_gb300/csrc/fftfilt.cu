// Overlap-add FFT filtering (include/filark.h, filark_fftfilt_*): the paper's
// benchmarked GPU filtering mode (Table 1, FFT-domain bandpass; Sec. 6.2,
// overlap-add chunked filtering), as a streaming operator with the chain's
// contract: y[n] = sum_{k<M} h[k] x[n-k], x before the stream start zero, the
// overlap tail carried across pushes.
//
// Each push is cut into blocks of at most L samples per channel.  A block b
// of len samples gives z = x_b * h (length len + M - 1) through an FFT of size
// N >= L + M - 1: Z = FFT(x_b) . H, z = IFFT(Z).  The outputs of the block are
// z[0, len) + tail[0, len); the tail becomes tail[len, ...) + z[len, ...).
// Two channels share one complex transform (x1 + i x2; h is real, so the
// real and imaginary parts of the result are the two convolutions).
//
// FFT: Stockham autosort in shared memory, one CTA per channel pair and
// block.  The log2(N) radix-2 steps are grouped into passes of radix 8 (one
// radix 2 or radix 4 pass first when log2(N) is not a multiple of 3); each
// thread does whole radix-R butterflies in registers.  The first forward pass
// reads the input block straight from global memory, the last forward pass
// multiplies by H, and the last inverse pass writes the outputs and the new
// tail straight to global memory.  The tail is double-buffered (read from one
// buffer, written to the other), so the epilogue needs no barrier.  Twiddles
// come from a host table made in double precision, one run of m values per
// pass (w_j = exp(-2 pi i j / (R m)), j < m, contiguous in j so that a warp
// reads consecutive entries), staged in shared memory; a butterfly's powers
// w^2 .. w^7 are products of at most three table values' roundings.  Shared arrays are padded by one element per 16 (element i at
// i + i/16), which spreads the strided stores of the early passes over the
// banks.  N <= 8192 (2 x 68 KB of complex floats plus 32 KB of twiddles).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "filark_internal.h"

using namespace filark;

namespace {

constexpr int kFftMaxThreads = 1024;
constexpr int kFftMaxLog = 13;     // N <= 8192

// padded shared-memory position of element i
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

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

struct FftParams {
    int N, logN, L, M;
    int twlen;          // entries of the per-pass twiddle table (<= N / 2)
    float scale;        // 1 / N
};

// Where a pass reads from and writes to.
enum { SRC_SMEM = 0, SRC_GIN = 1 };
enum { DST_SMEM = 0, DST_SMEM_H = 1, DST_GOUT = 2 };

struct BlockIO {
    const float *x;         // input block, time-major, row stride ldx
    long long ldx;
    int len;                // samples in this block
    int c1;                 // first channel of the pair (c1 + 1 the second, if has2)
    bool has2;
    const float2 *H;        // [N] spectrum of the taps
    const float *told;      // [C][M-1] tail before this block (NULL if M = 1)
    float *tnew;            // [C][M-1] tail after this block
    float *y;               // output block, row stride ldy
    long long ldy;
    int T1;                 // M - 1
    float scale;
};

// One Stockham pass of radix R: sub-transforms of length m = 2^logm are
// combined R at a time.  Butterfly t (< N/R) reads elements t + r N/R, scales
// them by w^r with w = exp(d 2 pi i j / (R m)) = tw[j] (this pass's run of
// the table), j = t mod m, and writes the radix-R DFT to (t - j) R + j + q m.
template <int R, bool INV, int SRC, int DST>
__device__ __forceinline__ void radix_pass(const float2 *__restrict__ a, float2 *__restrict__ b, int logN, int logm,
                                           const float2 *tw, const BlockIO &io) {
    constexpr int logR = R == 2 ? 1 : (R == 4 ? 2 : 3);
    const int N = 1 << logN, stride = N >> logR, m = 1 << logm;
    for (int t = threadIdx.x; t < stride; t += blockDim.x) {
        const int j = t & (m - 1);
        // the old tail values this butterfly's outputs add (issued first: they
        // do not depend on the transform)
        float2 told_q[DST == DST_GOUT ? R : 1];
        if constexpr (DST == DST_GOUT) {
            const int base = ((t - j) << logR) + j;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = base + (q << logm);
                told_q[q] = make_float2(0.f, 0.f);
                if (i < io.T1) {
                    told_q[q].x = __ldg(io.told + (long long)io.c1 * io.T1 + i);
                    if (io.has2) told_q[q].y = __ldg(io.told + (long long)(io.c1 + 1) * io.T1 + i);
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
                    re = __ldg(io.x + (long long)i * io.ldx + io.c1);
                    if (io.has2) im = __ldg(io.x + (long long)i * io.ldx + io.c1 + 1);
                }
                x[r] = make_float2(re, im);
            } else {
                x[r] = a[pad(i)];
            }
        }
        if (logm > 0) {
            float2 w = tw[j];
            if (INV) w.y = -w.y;
            if constexpr (R == 2) {
                x[1] = cmul(x[1], w);
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
        dft<R, INV>(x);
        const int base = ((t - j) << logR) + j;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = base + (q << logm);
            if constexpr (DST == DST_SMEM) {
                b[pad(i)] = x[q];
            } else if constexpr (DST == DST_SMEM_H) {
                b[pad(i)] = cmul(x[q], __ldg(io.H + i));
            } else {
                // z[i] (scaled) plus the old tail gives output i (i < len) or
                // new tail entry i - len (len <= i < len + M - 1)
                if (i < io.len + io.T1) {
                    const float v1 = x[q].x * io.scale + told_q[q].x, v2 = x[q].y * io.scale + told_q[q].y;
                    if (i < io.len) {
                        io.y[(long long)i * io.ldy + io.c1] = v1;
                        if (io.has2) io.y[(long long)i * io.ldy + io.c1 + 1] = v2;
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
__device__ __forceinline__ void radix_pass_any(int logR, const float2 *a, float2 *b, int logN, int logm,
                                               const float2 *tw, const BlockIO &io) {
    if (logR == 1) radix_pass<2, INV, SRC, DST>(a, b, logN, logm, tw, io);
    else if (logR == 2) radix_pass<4, INV, SRC, DST>(a, b, logN, logm, tw, io);
    else radix_pass<8, INV, SRC, DST>(a, b, logN, logm, tw, io);
}

// Forward transform of the input block (read from global memory), times H
// when io.H is set; the result is left in the returned buffer.
__device__ float2 *fft_forward(float2 *a, float2 *b, int logN, const float2 *tw, const BlockIO &io) {
    const int rem = logN % 3, npass = logN / 3 + (rem ? 1 : 0);
    int logm = 0, toff = 0;
    for (int p = 0; p < npass; ++p) {
        const int logR = (p == 0 && rem) ? rem : 3;
        const bool last = p == npass - 1;
        const float2 *twp = tw + toff;
        if (p == 0) {
            if (last && io.H) radix_pass_any<false, SRC_GIN, DST_SMEM_H>(logR, a, b, logN, logm, twp, io);
            else radix_pass_any<false, SRC_GIN, DST_SMEM>(logR, a, b, logN, logm, twp, io);
        } else {
            if (last && io.H) radix_pass_any<false, SRC_SMEM, DST_SMEM_H>(logR, a, b, logN, logm, twp, io);
            else radix_pass_any<false, SRC_SMEM, DST_SMEM>(logR, a, b, logN, logm, twp, io);
        }
        __syncthreads();
        float2 *tmp = a;
        a = b;
        b = tmp;
        if (logm > 0) toff += 1 << logm;
        logm += logR;
    }
    return a;
}

// Inverse transform of a (unscaled); the last pass writes outputs and tail.
__device__ void fft_inverse_out(float2 *a, float2 *b, int logN, const float2 *tw, const BlockIO &io) {
    const int rem = logN % 3, npass = logN / 3 + (rem ? 1 : 0);
    int logm = 0, toff = 0;
    for (int p = 0; p < npass; ++p) {
        const int logR = (p == 0 && rem) ? rem : 3;
        if (p == npass - 1) {
            radix_pass_any<true, SRC_SMEM, DST_GOUT>(logR, a, b, logN, logm, tw + toff, io);
        } else {
            radix_pass_any<true, SRC_SMEM, DST_SMEM>(logR, a, b, logN, logm, tw + toff, io);
            __syncthreads();
            float2 *tmp = a;
            a = b;
            b = tmp;
        }
        if (logm > 0) toff += 1 << logm;
        logm += logR;
    }
}

int fft_threads(int N) { return std::max(64, std::min(kFftMaxThreads, N / 8)); }

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
    io.H = H;
    io.told = told;
    io.tnew = tnew;
    io.y = y;
    io.ldy = ldy;
    io.T1 = fp.M - 1;
    io.scale = fp.scale;
    __syncthreads();
    float2 *X = fft_forward(sm, sm + NP, fp.logN, stw, io);
    fft_inverse_out(X, X == sm ? sm + NP : sm, fp.logN, stw, io);
}

__global__ void __launch_bounds__(kFftMaxThreads) fft_of_taps_kernel(const __grid_constant__ FftParams fp,
                                                                     const float *__restrict__ h,
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
    io.len = fp.M;
    io.c1 = 0;
    io.has2 = false;
    io.H = nullptr;
    const float2 *r = fft_forward(sm, sm + NP, fp.logN, stw, io);
    for (int i = threadIdx.x; i < fp.N; i += blockDim.x) H[i] = r[pad(i)];
}




// two padded buffers and the twiddle table
size_t fft_smem(int N) { return sizeof(float2) * (2 * (size_t)(N + (N >> 4)) + (size_t)(N / 2)); }

}  // namespace

struct filark_fftfilt {
    int device = 0, C = 0;
    long long max_chunk = 0;
    FftParams fp{};
    float2 *H = nullptr;
    float2 *tw = nullptr;       // exp(-2 pi i k / N), k < N/2
    float *tail[2] = {nullptr, nullptr};   // [C][M-1] each; tail[cur] is current
    int cur = 0;
};

extern "C" {

filark_status filark_fftfilt_create(int n_channels, int n_taps, const double *taps, int block_len,
                                    int64_t max_chunk, int cuda_device, filark_fftfilt **out) {
    if (!out) return fail_with(FILARK_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_channels < 1 || n_taps < 1 || !taps || max_chunk < 1)
        return fail_with(FILARK_EINVAL, "need n_channels >= 1, n_taps >= 1, taps, max_chunk >= 1");
    for (int k = 0; k < n_taps; ++k)
        if (!std::isfinite(taps[k])) return fail_with(FILARK_EINVAL, "non-finite tap");
    int L = block_len;
    if (L <= 0) {
        // default: the largest power-of-two block with N = 2 next_pow2(M) or more
        int n = 1;
        while (n < 2 * n_taps) n <<= 1;
        L = n - n_taps + 1;
    }
    int logN = 0;
    while ((1 << logN) < L + n_taps - 1) ++logN;
    if (logN > kFftMaxLog) return fail_with(FILARK_ENOSYS, "block_len + n_taps - 1 above the 8192-point FFT");
    filark_fftfilt *f = new (std::nothrow) filark_fftfilt();
    if (!f) return fail_with(FILARK_ENOMEM, "host allocation failed");
    f->device = cuda_device;
    f->C = n_channels;
    f->max_chunk = max_chunk;
    f->fp.logN = logN;
    f->fp.N = 1 << logN;
    f->fp.L = L;
    f->fp.M = n_taps;
    f->fp.scale = 1.0f / (float)f->fp.N;
    DeviceGuard dg(cuda_device);
    if (!dg.ok) {
        delete f;
        return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    }
    std::vector<float> hf((size_t)n_taps);
    for (int k = 0; k < n_taps; ++k) hf[(size_t)k] = (float)taps[k];
    // per-pass twiddle runs, in the kernels' pass order: w_j = exp(-2 pi i j / (R m)), j < m
    std::vector<float2> twh;
    {
        const int rem = logN % 3, npass = logN / 3 + (rem ? 1 : 0);
        int logm = 0;
        for (int p = 0; p < npass; ++p) {
            const int logR = (p == 0 && rem) ? rem : 3;
            if (logm > 0) {
                const int m = 1 << logm, Rm = m << logR;
                for (int j = 0; j < m; ++j) {
                    const double ang = -2.0 * 3.14159265358979323846 * (double)j / (double)Rm;
                    twh.push_back(make_float2((float)std::cos(ang), (float)std::sin(ang)));
                }
            }
            logm += logR;
        }
    }
    if (twh.empty()) twh.push_back(make_float2(1.f, 0.f));
    f->fp.twlen = (int)twh.size();
    float *dh = nullptr;
    cudaError_t e = cudaMalloc(&f->H, sizeof(float2) * (size_t)f->fp.N);
    if (e == cudaSuccess) e = cudaMalloc(&f->tw, sizeof(float2) * twh.size());
    if (e == cudaSuccess) e = cudaMemcpy(f->tw, twh.data(), sizeof(float2) * twh.size(), cudaMemcpyHostToDevice);
    const size_t tail_bytes = sizeof(float) * (size_t)n_channels * (size_t)(n_taps - 1);
    if (e == cudaSuccess && n_taps > 1) e = cudaMalloc(&f->tail[0], tail_bytes);
    if (e == cudaSuccess && n_taps > 1) e = cudaMalloc(&f->tail[1], tail_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&dh, sizeof(float) * (size_t)n_taps);
    if (e == cudaSuccess) e = cudaMemcpy(dh, hf.data(), sizeof(float) * hf.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fftfilt_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fft_smem(1 << kFftMaxLog));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft_of_taps_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fft_smem(1 << kFftMaxLog));
    if (e == cudaSuccess) {
        fft_of_taps_kernel<<<1, fft_threads(f->fp.N), fft_smem(f->fp.N)>>>(f->fp, dh, f->tw, f->H);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && f->tail[0]) e = cudaMemset(f->tail[0], 0, tail_bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (dh) cudaFree(dh);
    if (e != cudaSuccess) {
        if (f->H) cudaFree(f->H);
        if (f->tw) cudaFree(f->tw);
        if (f->tail[0]) cudaFree(f->tail[0]);
        if (f->tail[1]) cudaFree(f->tail[1]);
        delete f;
        return fail_cuda_with(e, "fftfilt create");
    }
    *out = f;
    return FILARK_OK;
}

filark_status filark_fftfilt_push(filark_fftfilt *f, const float *d_in, int64_t ld_in, int64_t n_samples,
                                  float *d_out, int64_t ld_out, filark_stream_t stream) {
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
    for (int64_t t = 0; t < n_samples; t += f->fp.L) {
        const int len = (int)std::min<int64_t>(f->fp.L, n_samples - t);
        fftfilt_block_kernel<<<pairs, fft_threads(f->fp.N), fft_smem(f->fp.N), s>>>(
            f->fp, d_in + t * ld_in, ld_in, len, f->C, f->H, f->tw, f->tail[f->cur], f->tail[1 - f->cur],
            d_out + t * ld_out, ld_out);
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
    const cudaError_t e = cudaMemsetAsync(f->tail[f->cur], 0, sizeof(float) * (size_t)f->C * (f->fp.M - 1),
                                          (cudaStream_t)stream);
    return e == cudaSuccess ? FILARK_OK : fail_cuda_with(e, "fftfilt reset");
}

filark_status filark_fftfilt_get_info(const filark_fftfilt *f, int *fft_len, int *block_len) {
    if (!f) return fail_with(FILARK_EINVAL, "filter is NULL");
    if (fft_len) *fft_len = f->fp.N;
    if (block_len) *block_len = f->fp.L;
    return FILARK_OK;
}

filark_status filark_fftfilt_destroy(filark_fftfilt *f) {
    if (!f) return FILARK_OK;
    DeviceGuard dg(f->device);
    cudaDeviceSynchronize();
    if (f->H) cudaFree(f->H);
    if (f->tw) cudaFree(f->tw);
    if (f->tail[0]) cudaFree(f->tail[0]);
    if (f->tail[1]) cudaFree(f->tail[1]);
    delete f;
    return FILARK_OK;
}

}  // extern "C"
