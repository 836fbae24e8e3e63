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
// FFT: radix-2 Stockham in shared memory, one CTA per channel pair and block,
// log2(N) passes of N/2 butterflies, twiddles from a table made on the host in
// double precision.  N <= 8192 (64 KB of complex floats, double-buffered in
// 128 KB of shared memory).
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "filark_internal.h"

using namespace filark;

namespace {

constexpr int kFftThreads = 512;
constexpr int kFftMaxLog = 13;     // N <= 8192

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Stockham radix-2 FFT of length N = 2^logN on buffers a <-> b in shared
// memory; inverse = false: exp(-i...) (forward), true: exp(+i...) (unscaled).
// tw[k] = exp(-2 pi i k / N), k < N/2.  Returns the buffer that holds the
// result.  All threads of the CTA call it.
__device__ float2 *fft_stockham(float2 *a, float2 *b, int logN, bool inverse, const float2 *__restrict__ tw) {
    const int N = 1 << logN, half = N >> 1;
    for (int s = 0; s < logN; ++s) {
        const int m = 1 << s;           // length of the sub-transforms already done
        for (int t = threadIdx.x; t < half; t += blockDim.x) {
            const int j = t & (m - 1);  // position inside the sub-transform
            const int k = t >> s;       // which pair of sub-transforms
            // twiddle exp(-+ i pi j / m) = tw[j N / (2m)]
            float2 w = __ldg(tw + (j << (logN - 1 - s)));
            if (inverse) w.y = -w.y;
            const float2 u = a[t];
            const float2 v = cmul(w, a[t + half]);
            b[2 * k * m + j] = make_float2(u.x + v.x, u.y + v.y);
            b[2 * k * m + j + m] = make_float2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
        float2 *tmp = a;
        a = b;
        b = tmp;
    }
    return a;
}

struct FftParams {
    int N, logN, L, M;
    float scale;        // 1 / N
};

// One CTA per (channel pair, block) of a launch; the blocks of one launch are
// consecutive and independent given the tail, so a launch covers exactly one
// block per channel pair and the host launches the blocks of a push in order.
__global__ void __launch_bounds__(kFftThreads) fftfilt_block_kernel(const __grid_constant__ FftParams fp,
                                                                    const float *__restrict__ x, long long ldx,
                                                                    int len, int C,
                                                                    const float2 *__restrict__ H,
                                                                    const float2 *__restrict__ tw,
                                                                    float *__restrict__ tail,   // [C][M-1]
                                                                    float *__restrict__ y, long long ldy) {
    extern __shared__ float2 sm[];
    float2 *a = sm, *b = sm + fp.N;
    const int c1 = 2 * blockIdx.x, c2 = c1 + 1;
    const bool has2 = c2 < C;
    for (int i = threadIdx.x; i < fp.N; i += blockDim.x) {
        float re = 0.f, im = 0.f;
        if (i < len) {
            re = x[(long long)i * ldx + c1];
            if (has2) im = x[(long long)i * ldx + c2];
        }
        a[i] = make_float2(re, im);
    }
    __syncthreads();
    float2 *X = fft_stockham(a, b, fp.logN, false, tw);
    float2 *other = X == a ? b : a;
    for (int i = threadIdx.x; i < fp.N; i += blockDim.x) X[i] = cmul(X[i], H[i]);
    __syncthreads();
    float2 *z = fft_stockham(X, other, fp.logN, true, tw);
    const int T1 = fp.M - 1;
    // outputs, then the new tail (each index is read before it is written:
    // outputs read tail[i] for i < len, the new tail entry i reads tail[i+len])
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const float2 v = z[i];
        const float t1 = i < T1 ? tail[(long long)c1 * T1 + i] : 0.f;
        y[(long long)i * ldy + c1] = v.x * fp.scale + t1;
        if (has2) {
            const float t2 = i < T1 ? tail[(long long)c2 * T1 + i] : 0.f;
            y[(long long)i * ldy + c2] = v.y * fp.scale + t2;
        }
    }
    __syncthreads();
    // new tail in registers first (in-place shift), then stored
    for (int base = 0; base < T1; base += blockDim.x) {
        const int i = base + threadIdx.x;
        float n1 = 0.f, n2 = 0.f;
        if (i < T1) {
            const float2 v = z[len + i];
            n1 = v.x * fp.scale + (i + len < T1 ? tail[(long long)c1 * T1 + i + len] : 0.f);
            if (has2) n2 = v.y * fp.scale + (i + len < T1 ? tail[(long long)c2 * T1 + i + len] : 0.f);
        }
        __syncthreads();
        if (i < T1) {
            tail[(long long)c1 * T1 + i] = n1;
            if (has2) tail[(long long)c2 * T1 + i] = n2;
        }
        __syncthreads();
    }
}

__global__ void fft_of_taps_kernel(const __grid_constant__ FftParams fp, const float *__restrict__ h,
                                   const float2 *__restrict__ tw, float2 *__restrict__ H) {
    extern __shared__ float2 sm[];
    float2 *a = sm, *b = sm + fp.N;
    for (int i = threadIdx.x; i < fp.N; i += blockDim.x) a[i] = make_float2(i < fp.M ? h[i] : 0.f, 0.f);
    __syncthreads();
    float2 *r = fft_stockham(a, b, fp.logN, false, tw);
    for (int i = threadIdx.x; i < fp.N; i += blockDim.x) H[i] = r[i];
}

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

filark_status ffail(filark_status st, const std::string &m) {
    set_last_error(m);
    return st;
}

filark_status fcuda(cudaError_t e, const char *what) {
    cudaGetLastError();
    set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    return FILARK_ECUDA;
}

size_t fft_smem(int N) { return sizeof(float2) * 2 * (size_t)N; }

}  // namespace

struct filark_fftfilt {
    int device = 0, C = 0;
    long long max_chunk = 0;
    FftParams fp{};
    float2 *H = nullptr;
    float2 *tw = nullptr;       // exp(-2 pi i k / N), k < N/2
    float *tail = nullptr;
};

extern "C" {

filark_status filark_fftfilt_create(int n_channels, int n_taps, const double *taps, int block_len,
                                    int64_t max_chunk, int cuda_device, filark_fftfilt **out) {
    if (!out) return ffail(FILARK_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_channels < 1 || n_taps < 1 || !taps || max_chunk < 1)
        return ffail(FILARK_EINVAL, "need n_channels >= 1, n_taps >= 1, taps, max_chunk >= 1");
    for (int k = 0; k < n_taps; ++k)
        if (!std::isfinite(taps[k])) return ffail(FILARK_EINVAL, "non-finite tap");
    int L = block_len;
    if (L <= 0) {
        // default: the largest power-of-two block with N = 2 next_pow2(M) or more
        int n = 1;
        while (n < 2 * n_taps) n <<= 1;
        L = n - n_taps + 1;
    }
    int logN = 0;
    while ((1 << logN) < L + n_taps - 1) ++logN;
    if (logN > kFftMaxLog) return ffail(FILARK_ENOSYS, "block_len + n_taps - 1 above the 8192-point FFT");
    filark_fftfilt *f = new (std::nothrow) filark_fftfilt();
    if (!f) return ffail(FILARK_ENOMEM, "host allocation failed");
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
        return ffail(FILARK_ECUDA, "cudaSetDevice failed");
    }
    std::vector<float> hf((size_t)n_taps);
    for (int k = 0; k < n_taps; ++k) hf[(size_t)k] = (float)taps[k];
    std::vector<float2> twh((size_t)f->fp.N / 2);
    for (int k = 0; k < f->fp.N / 2; ++k) {
        const double ang = -2.0 * 3.14159265358979323846 * (double)k / (double)f->fp.N;
        twh[(size_t)k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    float *dh = nullptr;
    cudaError_t e = cudaMalloc(&f->H, sizeof(float2) * (size_t)f->fp.N);
    if (e == cudaSuccess) e = cudaMalloc(&f->tw, sizeof(float2) * twh.size());
    if (e == cudaSuccess) e = cudaMemcpy(f->tw, twh.data(), sizeof(float2) * twh.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n_taps > 1) e = cudaMalloc(&f->tail, sizeof(float) * (size_t)n_channels * (n_taps - 1));
    if (e == cudaSuccess) e = cudaMalloc(&dh, sizeof(float) * (size_t)n_taps);
    if (e == cudaSuccess) e = cudaMemcpy(dh, hf.data(), sizeof(float) * hf.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fftfilt_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fft_smem(1 << kFftMaxLog));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft_of_taps_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fft_smem(1 << kFftMaxLog));
    if (e == cudaSuccess) {
        fft_of_taps_kernel<<<1, kFftThreads, fft_smem(f->fp.N)>>>(f->fp, dh, f->tw, f->H);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && f->tail) e = cudaMemset(f->tail, 0, sizeof(float) * (size_t)n_channels * (n_taps - 1));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (dh) cudaFree(dh);
    if (e != cudaSuccess) {
        if (f->H) cudaFree(f->H);
        if (f->tw) cudaFree(f->tw);
        if (f->tail) cudaFree(f->tail);
        delete f;
        return fcuda(e, "fftfilt create");
    }
    *out = f;
    return FILARK_OK;
}

filark_status filark_fftfilt_push(filark_fftfilt *f, const float *d_in, int64_t ld_in, int64_t n_samples,
                                  float *d_out, int64_t ld_out, filark_stream_t stream) {
    if (!f) return ffail(FILARK_EINVAL, "filter is NULL");
    if (n_samples < 0 || n_samples > f->max_chunk) return ffail(FILARK_EINVAL, "n_samples must be in [0, max_chunk]");
    if (n_samples == 0) return FILARK_OK;
    if (!d_in || !d_out || ld_in < f->C || ld_out < f->C) return ffail(FILARK_EINVAL, "buffers NULL or ld < C");
    const size_t in_bytes = sizeof(float) * (size_t)((n_samples - 1) * ld_in + f->C);
    const size_t out_bytes = sizeof(float) * (size_t)((n_samples - 1) * ld_out + f->C);
    const char *pi = (const char *)d_in, *po = (const char *)d_out;
    if (pi < po + out_bytes && po < pi + in_bytes) return ffail(FILARK_EINVAL, "output overlaps the input");
    DeviceGuard dg(f->device);
    if (!dg.ok) return ffail(FILARK_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned pairs = (unsigned)((f->C + 1) / 2);
    for (int64_t t = 0; t < n_samples; t += f->fp.L) {
        const int len = (int)std::min<int64_t>(f->fp.L, n_samples - t);
        fftfilt_block_kernel<<<pairs, kFftThreads, fft_smem(f->fp.N), s>>>(f->fp, d_in + t * ld_in, ld_in, len, f->C,
                                                                           f->H, f->tw, f->tail, d_out + t * ld_out,
                                                                           ld_out);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FILARK_OK : fcuda(e, "fftfilt push");
}

filark_status filark_fftfilt_reset(filark_fftfilt *f, filark_stream_t stream) {
    if (!f) return ffail(FILARK_EINVAL, "filter is NULL");
    DeviceGuard dg(f->device);
    if (!dg.ok) return ffail(FILARK_ECUDA, "cudaSetDevice failed");
    if (!f->tail) return FILARK_OK;
    const cudaError_t e = cudaMemsetAsync(f->tail, 0, sizeof(float) * (size_t)f->C * (f->fp.M - 1),
                                          (cudaStream_t)stream);
    return e == cudaSuccess ? FILARK_OK : fcuda(e, "fftfilt reset");
}

filark_status filark_fftfilt_get_info(const filark_fftfilt *f, int *fft_len, int *block_len) {
    if (!f) return ffail(FILARK_EINVAL, "filter is NULL");
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
    if (f->tail) cudaFree(f->tail);
    delete f;
    return FILARK_OK;
}

}  // extern "C"
