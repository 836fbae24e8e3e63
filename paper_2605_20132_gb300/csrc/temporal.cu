// Stateful temporal operators on the chain's streaming contract
// (include/filark.h, filark_top_*): the concatenation of the outputs of any
// sequence of pushes equals one push of the whole recording, x before the
// stream start is zero (Sec. 3.4, stateful-compatible operators; Table 1,
// temporal filters and amplitude operators).
//
//   FIR   y[n] = sum_{k<M} h[k] x[n-k]: the last M-1 inputs of every channel
//         are carried (overlap-save).  CTA = 32 channels x 256 outputs; the
//         inputs with M-1 rows of history sit in shared memory; each thread
//         makes 32 consecutive outputs of one channel from a 63-value register
//         window per 32 taps, the last M mod 32 taps in groups of 8 (FFMA with
//         the taps as constant-bank operands).
//   MEAN  y[n] = (1/w) sum_{k<w} x[n-k]
//   AGC   g[n] = (1/w) sum_{k<w} |x[n-k]|, y[n] = x[n] / g[n] (0 if g = 0)
//         Window sums are differences of a running prefix P of x (or |x|) kept
//         in double-float (~48 bits) in a ring of w + max_chunk rows: a prefix
//         kernel (one CTA per 8 channels walks the push in slabs of 32 blocks
//         x 32 samples: block sums, per-channel prefix over the blocks, the
//         samples' prefixes) and an output kernel over all samples.
//   EMA   e[n] = (1-a) e[n-1] + a x[n]^2, y[n] = x[n] / sqrt(e[n]) (0 if e = 0)
//         One CTA per 16 channels x 32 time segments; a push is one slab of
//         32 segments of ceil(T / 32) samples (<= 64; longer pushes take
//         several slabs), so every SM holds several CTAs and the push is one
//         wave.  Per segment the response from a zero start (FP32), segment
//         starts from the carried state through the powers (1-a)^(seg j), the
//         carried state itself in double-float; the input is read twice
//         (the second time from L2) instead of being held in registers.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>

#include "filark_internal.h"
#include "host_trace.h"

using namespace filark;

namespace {

constexpr int kTopCh = 32;          // channels per CTA
constexpr int kFirRows = 256;       // FIR outputs per CTA
constexpr int kFirThreads = 256;    // (channel, group of 32 outputs)
constexpr int kFirMaxTaps = 512;
constexpr int kScanBlocks = 32;     // blocks of 32 samples per slab (window / EMA kernels)
constexpr int kScanCh = 8;          // channels per CTA of the prefix kernel: 32-byte rows,
                                    // and enough CTAs (C / 8) to fill every SM
constexpr int kScanThreads = kScanCh * kScanBlocks;  // 256
constexpr int kSlab = 32 * kScanBlocks;              // 1024 samples
constexpr int kEmaCh = 16;          // channels per CTA of the EMA kernel
constexpr int kEmaSegs = 32;        // time segments per slab
constexpr int kEmaThreads = kEmaCh * kEmaSegs;       // 512
constexpr int kEmaMaxSeg = 64;      // samples per segment at most (slabs <= 2048 samples)

struct DF2 {
    float hi, lo;
};
__device__ __forceinline__ DF2 d_add(DF2 a, DF2 b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float err = (a.hi - (s - bb)) + (b.hi - bb);
    const float lo = err + (a.lo + b.lo);
    const float hi = s + lo;
    return DF2{hi, lo - (hi - s)};
}
__device__ __forceinline__ DF2 d_add_f(DF2 a, float b) { return d_add(a, DF2{b, 0.f}); }
__device__ __forceinline__ DF2 d_mul(DF2 a, DF2 b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float hi = p + e;
    return DF2{hi, e - (hi - p)};
}

// ------------------------------------------------------------------- FIR --

struct FirParams {
    float h[kFirMaxTaps];   // taps, zero past M
    int M, Mpad;            // taps; taps rounded up to 32
};

// history: [M-1][ldh] floats, row j = sample (push start - (M-1) + j)
__global__ void __launch_bounds__(kFirThreads) fir_kernel(const __grid_constant__ FirParams fp,
                                                          const float *__restrict__ x, long long ldx, int T, int C,
                                                          const float *__restrict__ hist,
                                                          float *__restrict__ y, long long ldy) {
    extern __shared__ float xs[];   // [Mpad + kFirRows][kTopCh]; row OFF + r = input row t0 + r
    const int OFF = fp.Mpad;
    const int c0 = blockIdx.x * kTopCh, t0 = blockIdx.y * kFirRows;
    const int tid = threadIdx.x;
    const int nrows = OFF + kFirRows;
    // 16-byte loads when every row of input and history starts 16-byte aligned
    const bool vec4 = ((ldx | C) & 3) == 0 && (((uintptr_t)x | (uintptr_t)hist) & 15) == 0;
    if (vec4) {
        // asynchronous 16-byte copies, all in flight together; quads out of
        // range are zero-filled (source size 0)
        for (int f = tid; f < nrows * (kTopCh / 4); f += kFirThreads) {
            const int s = f / (kTopCh / 4), q = f % (kTopCh / 4);
            const int r = s - OFF;
            const long long g = (long long)t0 + r;
            const int c = c0 + 4 * q;
            const bool in = c < C && r > -fp.M && g < T;   // C % 4 == 0: the whole quad is in range
            const float *src = !in ? x : (g >= 0 ? x + g * ldx + c : hist + (g + fp.M - 1) * (long long)C + c);
            const unsigned dst = (unsigned)__cvta_generic_to_shared(&xs[s * kTopCh + 4 * q]);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(in ? 16 : 0)
                         : "memory");
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    } else {
        for (int f = tid; f < nrows * kTopCh; f += kFirThreads) {
            const int s = f / kTopCh, ch = f % kTopCh;
            const int r = s - OFF;                 // tile row, negative = earlier
            const long long g = (long long)t0 + r;  // sample index within the push
            const int c = c0 + ch;
            float v = 0.f;
            if (c < C && r > -fp.M && g < T) {
                if (g >= 0) v = __ldg(x + g * ldx + c);
                else v = __ldg(hist + (g + fp.M - 1) * (long long)C + c);
            }
            xs[f] = v;
        }
    }
    __syncthreads();
    const int ch = tid & 31, r0 = (tid >> 5) * 32;
    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    const int M32 = fp.M & ~31;
    for (int k0 = 0; k0 < M32; k0 += 32) {
        // w[q] = input row r0 - k0 - 31 + q, q = 0..62
        float w[63];
        const float *base = xs + (OFF + r0 - k0 - 31) * kTopCh + ch;
#pragma unroll
        for (int q = 0; q < 63; ++q) w[q] = base[q * kTopCh];
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) {
            const float hk = fp.h[k0 + kk];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = fmaf(hk, w[j - kk + 31], acc[j]);
        }
    }
    // the remaining taps in groups of 8 (the taps past M are zero)
    for (int k0 = M32; k0 < fp.M; k0 += 8) {
        // w[q] = input row r0 - k0 - 7 + q, q = 0..38
        float w[39];
        const float *base = xs + (OFF + r0 - k0 - 7) * kTopCh + ch;
#pragma unroll
        for (int q = 0; q < 39; ++q) w[q] = base[q * kTopCh];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const float hk = fp.h[k0 + kk];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = fmaf(hk, w[j - kk + 7], acc[j]);
        }
    }
    const int c = c0 + ch;
    if (c < C) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int g = t0 + r0 + j;
            if (g < T) y[(long long)g * ldy + c] = acc[j];
        }
    }
}

// next history = the last M-1 samples of (history, push); grid (channel
// groups of 256, history rows)
__global__ void fir_history_kernel(const float *__restrict__ x, long long ldx, int T, int C, int M,
                                   const float *__restrict__ hist, float *__restrict__ hist_next) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (c >= C) return;
    const long long src = (long long)j + T;   // position in (history, push)
    hist_next[(long long)j * C + c] = src >= M - 1 ? x[(src - (M - 1)) * ldx + c] : hist[src * C + c];
}

// ------------------------------------------------------ window sums (P) --

// One CTA per 8 channels walks the push in slabs of 1024 samples and writes
// the running prefix P[n] (double-float) of u = x (MEAN) or |x| (AGC).
// slot0 = n0 mod Q, the ring row of the push's first sample.
__global__ void __launch_bounds__(kScanThreads, 5) prefix_kernel(const float *__restrict__ x, long long ldx, int T,
                                                              int C, int absval, int slot0, int Q,
                                                              float2 *__restrict__ ring,
                                                              float2 *__restrict__ carry) {
    __shared__ DF2 bs[kScanBlocks][kScanCh];
    __shared__ DF2 cin[kScanCh];
    const int ch = threadIdx.x % kScanCh, blk = threadIdx.x / kScanCh;
    const int c = blockIdx.x * kScanCh + ch;
    if (blk == 0) cin[ch] = c < C ? DF2{carry[c].x, carry[c].y} : DF2{0.f, 0.f};
    __syncthreads();
    for (int s0 = 0; s0 < T; s0 += kSlab) {
        const int a = s0 + blk * 32;
        float u[32];
        DF2 sum{0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            float v = 0.f;
            if (c < C && a + i < T) v = x[(long long)(a + i) * ldx + c];
            u[i] = absval ? fabsf(v) : v;
            sum = d_add_f(sum, u[i]);
        }
        bs[blk][ch] = sum;
        __syncthreads();
        DF2 p = cin[ch];
        for (int j = 0; j < blk; ++j) p = d_add(p, bs[j][ch]);
        if (c < C && a < T) {
            int slot = slot0 + a;                // slot0 < Q and a < T < Q: at most one wrap
            if (slot >= Q) slot -= Q;
            float2 *rc = ring + c;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (a + i >= T) break;
                p = d_add_f(p, u[i]);
                rc[(size_t)slot * C] = make_float2(p.hi, p.lo);
                slot = slot + 1 == Q ? 0 : slot + 1;
            }
        }
        __syncthreads();
        if (blk == 0) {
            DF2 t = cin[ch];
            for (int j = 0; j < kScanBlocks; ++j) t = d_add(t, bs[j][ch]);
            cin[ch] = t;
        }
        __syncthreads();
    }
    if (blk == 0 && c < C) carry[c] = make_float2(cin[ch].hi, cin[ch].lo);
}

// grid (channel groups of 256, rows; rows past gridDim.y loop); slot0 = n0 mod Q
__global__ void window_out_kernel(const float *__restrict__ x, long long ldx, int T, int C, int w, int agc,
                                  long long n0, int slot0, int Q, const float2 *__restrict__ ring,
                                  float *__restrict__ y, long long ldy) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    for (int t = blockIdx.y; t < T; t += gridDim.y) {
        int sn = slot0 + t;                          // t < T < Q: at most one wrap
        if (sn >= Q) sn -= Q;
        const float2 pn = ring[(size_t)sn * C + c];
        float2 pw = make_float2(0.f, 0.f);
        if (n0 + t - w >= 0) {
            int sw = sn - w;                         // w < Q
            if (sw < 0) sw += Q;
            pw = ring[(size_t)sw * C + c];
        }
        const DF2 d = d_add(DF2{pn.x, pn.y}, DF2{-pw.x, -pw.y});
        const float g = (d.hi + d.lo) / (float)w;
        float out = g;
        if (agc) {
            const float v = x[(long long)t * ldx + c];
            out = g > 0.f ? v / g : 0.f;
        }
        y[(long long)t * ldy + c] = out;
    }
}

// ------------------------------------------------------------------- EMA --

struct EmaParams {
    float alpha;                  // a
    float ac, ac_lo;              // 1 - a as a float pair: a float alone would move
                                  // a slow EMA's time constant (1-a = 0.9999 to ~6e-8)
    int seg;                      // samples per segment for this push
    float pwseg[kEmaSegs + 1];    // (1-a)^(seg j), FP32
    float pw1[kEmaMaxSeg + 1];    // (1-a)^j, FP32
    float pslab_hi, pslab_lo;     // (1-a)^(32 seg), double-float (full slabs)
    float plast_hi, plast_lo;     // (1-a)^(length of the push's last slab), double-float
};

__global__ void __launch_bounds__(kEmaThreads, 3) ema_kernel(const __grid_constant__ EmaParams ep,
                                                              const float *__restrict__ x, long long ldx, int T,
                                                              int C, float2 *__restrict__ state,
                                                              float *__restrict__ y, long long ldy) {
    __shared__ float ls[kEmaSegs][kEmaCh];
    __shared__ DF2 es[kEmaCh];
    const int ch = threadIdx.x % kEmaCh, sg = threadIdx.x / kEmaCh;
    const int c = blockIdx.x * kEmaCh + ch;
    const int seg = ep.seg, slab_len = kEmaSegs * seg;
    if (sg == 0) es[ch] = c < C ? DF2{state[c].x, state[c].y} : DF2{0.f, 0.f};
    __syncthreads();
    for (int s0 = 0; s0 < T; s0 += slab_len) {
        const int slab = min(slab_len, T - s0);
        const int a = s0 + sg * seg;
        const int n_here = c < C ? max(0, min(seg, T - a)) : 0;   // samples of this segment
        const float *xp = x + (long long)a * ldx + c;
        // this segment's response at its last sample from a zero start (FP32)
        float l = 0.f;
#pragma unroll 8
        for (int i = 0; i < n_here; ++i) {
            const float v = __ldg(xp + (long long)i * ldx);
            l = fmaf(ep.ac, l, fmaf(ep.ac_lo, l, ep.alpha * v * v));
        }
        ls[sg][ch] = l;
        __syncthreads();
        // start of this segment: (1-a)^(seg sg) E + sum_{j<sg} (1-a)^(seg (sg-1-j)) l_j
        const DF2 E = es[ch];
        float e = ep.pwseg[sg] * E.hi;
        for (int j = 0; j < sg; ++j) e = fmaf(ep.pwseg[sg - 1 - j], ls[j][ch], e);
        float *yp = y + (long long)a * ldy + c;
#pragma unroll 8
        for (int i = 0; i < n_here; ++i) {
            const float v = __ldg(xp + (long long)i * ldx);
            e = fmaf(ep.ac, e, fmaf(ep.ac_lo, e, ep.alpha * v * v));
            yp[(long long)i * ldy] = e > 0.f ? v * rsqrtf(e) : 0.f;
        }
        __syncthreads();
        if (sg == 0) {
            // state after the slab's last sample, double-float:
            // (1-a)^slab E + sum_j (1-a)^(samples after segment j) l_j
            const int nb = (slab + seg - 1) / seg;
            const int tail = slab - seg * (nb - 1);      // samples of the last segment
            DF2 t = d_mul(E, slab == slab_len ? DF2{ep.pslab_hi, ep.pslab_lo} : DF2{ep.plast_hi, ep.plast_lo});
            float add = 0.f;
            for (int j = 0; j < nb; ++j) {
                const float pw = j < nb - 1 ? ep.pw1[tail] * ep.pwseg[nb - 2 - j] : 1.f;
                add = fmaf(pw, ls[j][ch], add);
            }
            es[ch] = d_add_f(t, add);
        }
        __syncthreads();
    }
    if (sg == 0 && c < C) state[c] = make_float2(es[ch].hi, es[ch].lo);
}

// ------------------------------------------------------------------ host --




size_t fir_smem(int Mpad) { return sizeof(float) * (size_t)(Mpad + kFirRows) * kTopCh; }

}  // namespace

struct filark_top {
    int kind = 0, device = 0, C = 0, M = 1;
    long long max_chunk = 0, n = 0;
    FirParams fir{};
    EmaParams ema{};
    float *hist[2] = {nullptr, nullptr};
    int parity = 0;
    float2 *ring = nullptr;
    long long Q = 0;
    float2 *carry = nullptr;   // window prefix or EMA state
};

namespace {

void free_top(filark_top *t) {
    if (!t) return;
    for (float *p : t->hist)
        if (p) cudaFree(p);
    if (t->ring) cudaFree(t->ring);
    if (t->carry) cudaFree(t->carry);
    delete t;
}

filark_status zero_top(filark_top *t, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (float *p : t->hist)
        if (p && e == cudaSuccess) e = cudaMemsetAsync(p, 0, sizeof(float) * (size_t)(t->M - 1) * t->C, s);
    if (t->carry && e == cudaSuccess) e = cudaMemsetAsync(t->carry, 0, sizeof(float2) * (size_t)t->C, s);
    if (e != cudaSuccess) return fail_cuda_with(e, "temporal operator: reset");
    t->n = 0;
    t->parity = 0;
    return FILARK_OK;
}

}  // namespace

extern "C" {

filark_status filark_top_create(int kind, int n_channels, int length, const double *taps, double alpha,
                                int64_t max_chunk, int cuda_device, filark_top **out) {
    if (!out) return fail_with(FILARK_EINVAL, "out is NULL");
    *out = nullptr;
    if (kind < FILARK_TOP_FIR || kind > FILARK_TOP_EMA) return fail_with(FILARK_EINVAL, "unknown operator kind");
    if (n_channels < 1) return fail_with(FILARK_EINVAL, "n_channels must be >= 1");
    if (max_chunk < 1 || max_chunk > (int64_t)1 << 30) return fail_with(FILARK_EINVAL, "max_chunk out of range");
    filark_top *t = new (std::nothrow) filark_top();
    if (!t) return fail_with(FILARK_ENOMEM, "host allocation failed");
    t->kind = kind;
    t->device = cuda_device;
    t->C = n_channels;
    t->max_chunk = max_chunk;
    if (kind == FILARK_TOP_FIR) {
        if (length < 1 || length > kFirMaxTaps || !taps) {
            delete t;
            return fail_with(FILARK_EINVAL, "FIR needs 1 <= taps <= 512 and a taps array");
        }
        for (int k = 0; k < length; ++k)
            if (!std::isfinite(taps[k])) {
                delete t;
                return fail_with(FILARK_EINVAL, "non-finite tap");
            }
        t->M = length;
        t->fir.M = length;
        t->fir.Mpad = (length + 31) / 32 * 32;
        for (int k = 0; k < length; ++k) t->fir.h[k] = (float)taps[k];
    } else if (kind == FILARK_TOP_MEAN || kind == FILARK_TOP_AGC) {
        if (length < 1 || length > (1 << 24)) {
            delete t;
            return fail_with(FILARK_EINVAL, "window length must be in [1, 2^24]");
        }
        t->M = length;
        t->Q = (long long)length + max_chunk;
        if ((double)t->Q * n_channels > 2.0e9) {
            delete t;
            return fail_with(FILARK_ENOSYS, "window ring above 2^31 entries");
        }
    } else {
        if (!(alpha > 0.0) || !(alpha <= 1.0)) {
            delete t;
            return fail_with(FILARK_EINVAL, "EMA coefficient must be in (0, 1]");
        }
        t->M = 1;
        const double ac = 1.0 - alpha;
        t->ema.alpha = (float)alpha;
        t->ema.ac = (float)ac;
        t->ema.ac_lo = (float)(ac - (double)t->ema.ac);
        for (int j = 0; j <= kEmaMaxSeg; ++j) t->ema.pw1[j] = (float)std::pow(ac, (double)j);
        t->ema.seg = 0;   // segment tables filled at the first push
    }
    DeviceGuard dg(cuda_device);
    if (!dg.ok) {
        delete t;
        return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    }
    cudaError_t e = cudaSuccess;
    if (kind == FILARK_TOP_FIR) {
        if (t->M > 1)
            for (int k = 0; k < 2 && e == cudaSuccess; ++k)
                e = cudaMalloc(&t->hist[k], sizeof(float) * (size_t)(t->M - 1) * t->C);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fir_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fir_smem(kFirMaxTaps));
    } else {
        e = cudaMalloc(&t->carry, sizeof(float2) * (size_t)t->C);
        if (e == cudaSuccess && t->Q > 0) e = cudaMalloc(&t->ring, sizeof(float2) * (size_t)t->Q * t->C);
    }
    if (e != cudaSuccess) {
        free_top(t);
        return fail_cuda_with(e, "temporal operator create");
    }
    filark_status st = zero_top(t, nullptr);
    if (st == FILARK_OK && (e = cudaStreamSynchronize(nullptr)) != cudaSuccess) st = fail_cuda_with(e, "create: sync");
    if (st != FILARK_OK) {
        free_top(t);
        return st;
    }
    *out = t;
    return FILARK_OK;
}

filark_status filark_top_push(filark_top *t, const float *d_in, int64_t ld_in, int64_t n_samples, float *d_out,
                              int64_t ld_out, filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_top_push");
    if (!t) return fail_with(FILARK_EINVAL, "operator is NULL");
    if (n_samples < 0 || n_samples > t->max_chunk) return fail_with(FILARK_EINVAL, "n_samples must be in [0, max_chunk]");
    if (n_samples == 0) return FILARK_OK;
    if (!d_in || !d_out || ld_in < t->C || ld_out < t->C) return fail_with(FILARK_EINVAL, "buffers NULL or ld < C");
    const size_t in_bytes = sizeof(float) * (size_t)((n_samples - 1) * ld_in + t->C);
    const size_t out_bytes = sizeof(float) * (size_t)((n_samples - 1) * ld_out + t->C);
    const char *pi = (const char *)d_in, *po = (const char *)d_out;
    if (pi < po + out_bytes && po < pi + in_bytes) return fail_with(FILARK_EINVAL, "output overlaps the input");
    DeviceGuard dg(t->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    const int T = (int)n_samples, C = t->C;
    const unsigned gch = (unsigned)((C + kTopCh - 1) / kTopCh);
    const unsigned gscan = (unsigned)((C + kScanCh - 1) / kScanCh);
    if (t->kind == FILARK_TOP_FIR) {
        const dim3 grid(gch, (unsigned)((T + kFirRows - 1) / kFirRows));
        const float *h = t->M > 1 ? t->hist[t->parity] : nullptr;
        fir_kernel<<<grid, kFirThreads, fir_smem(t->fir.Mpad), s>>>(t->fir, d_in, ld_in, T, C, h, d_out, ld_out);
        if (t->M > 1) {
            const dim3 gh((unsigned)((C + 255) / 256), (unsigned)(t->M - 1));
            fir_history_kernel<<<gh, 256, 0, s>>>(d_in, ld_in, T, C, t->M, h, t->hist[t->parity ^ 1]);
            t->parity ^= 1;
        }
    } else if (t->kind == FILARK_TOP_MEAN || t->kind == FILARK_TOP_AGC) {
        const int agc = t->kind == FILARK_TOP_AGC;
        const int slot0 = (int)(t->n % t->Q);
        prefix_kernel<<<gscan, kScanThreads, 0, s>>>(d_in, ld_in, T, C, agc, slot0, (int)t->Q, t->ring, t->carry);
        const dim3 gout((unsigned)((C + 255) / 256), (unsigned)std::min(T, 65535));
        window_out_kernel<<<gout, 256, 0, s>>>(d_in, ld_in, T, C, t->M, agc, t->n, slot0, (int)t->Q, t->ring,
                                               d_out, ld_out);
    } else {
        // one slab of 32 segments per push where it fits in 32 x 64 samples
        const int seg = std::min(kEmaMaxSeg, (T + kEmaSegs - 1) / kEmaSegs);
        const double acd = (double)t->ema.ac + (double)t->ema.ac_lo;
        if (t->ema.seg != seg) {
            t->ema.seg = seg;
            for (int j = 0; j <= kEmaSegs; ++j) t->ema.pwseg[j] = (float)std::pow(acd, (double)seg * j);
            const double ps = std::pow(acd, (double)seg * kEmaSegs);
            t->ema.pslab_hi = (float)ps;
            t->ema.pslab_lo = (float)(ps - (double)t->ema.pslab_hi);
        }
        EmaParams ep = t->ema;
        const int slab_len = kEmaSegs * seg;
        const int last = T - (T - 1) / slab_len * slab_len;   // length of the last slab
        const double pl = std::pow(acd, (double)last);
        ep.plast_hi = (float)pl;
        ep.plast_lo = (float)(pl - (double)ep.plast_hi);
        ema_kernel<<<(unsigned)((C + kEmaCh - 1) / kEmaCh), kEmaThreads, 0, s>>>(ep, d_in, ld_in, T, C, t->carry, d_out, ld_out);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda_with(e, "temporal operator push");
    t->n += n_samples;
    return FILARK_OK;
}

filark_status filark_top_reset(filark_top *t, filark_stream_t stream) {
    if (!t) return fail_with(FILARK_EINVAL, "operator is NULL");
    DeviceGuard dg(t->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    return zero_top(t, (cudaStream_t)stream);
}

filark_status filark_top_destroy(filark_top *t) {
    if (!t) return FILARK_OK;
    DeviceGuard dg(t->device);
    cudaDeviceSynchronize();
    free_top(t);
    return FILARK_OK;
}

}  // extern "C"
