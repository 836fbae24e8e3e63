// Headless streaming display path (include/filark.h, filark_view_*): the
// paper's ring-buffer texture (Sec. 3.2, ring-buffer streaming visualization:
// fixed-size buffer, equal-width time slots, only the newly exposed region
// written, a ring offset for the logical start), view-dependent downsampling
// (Sec. 3.5: drop, peak and linear modes) and the render-time causal display
// filter with state kept across viewport updates -- as a device buffer, with
// no graphics API.
//
// A push of T samples x C channels:
//   1. channels -> H display rows (groups of kc channels) per sample;
//   2. optional causal SOS display filter on the rows at the source rate:
//      the chain of this library (bandpass stage only) with carried state;
//   3. samples -> display columns (groups of kt samples); the samples of the
//      incomplete last column are carried to the next push;
//   4. each completed column j is written to ring column j mod W -- only the
//      newly exposed columns move, whatever the length of the recording.
// filark_view_image unrolls the ring into [H][W], oldest column at the left.
#include <cstdint>
#include <cstring>
#include <new>
#include <string>

#include "filark_internal.h"
#include "host_trace.h"

using namespace filark;

namespace {

// one display value from n values at stride `st`: drop = the first, peak = the
// largest magnitude (first on ties), linear = interpolation at the centre
__device__ __forceinline__ float reduce_group(const float *p, long long st, int n, int mode) {
    if (mode == FILARK_VIEW_DROP || n == 1) return p[0];
    if (mode == FILARK_VIEW_PEAK) {
        float best = p[0], mag = fabsf(p[0]);
        int i = 1;
        // four loads in flight, then the comparisons in order (first on ties)
        for (; i + 4 <= n; i += 4) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = p[(long long)(i + u) * st];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (fabsf(v[u]) > mag) {
                    mag = fabsf(v[u]);
                    best = v[u];
                }
        }
        for (; i < n; ++i) {
            const float v = p[(long long)i * st];
            if (fabsf(v) > mag) {
                mag = fabsf(v);
                best = v;
            }
        }
        return best;
    }
    const int i0 = (n - 1) >> 1;
    if (n & 1) return p[(long long)i0 * st];
    return 0.5f * p[(long long)i0 * st] + 0.5f * p[(long long)(i0 + 1) * st];
}

// grid (row groups of 256, samples; samples past gridDim.y loop)
__global__ void view_rows_kernel(const float *__restrict__ x, long long ldx, int T, int C, int kc, int H, int mode,
                                 float *__restrict__ rows) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    const int c0 = r * kc, n = min(C, c0 + kc) - c0;
#pragma unroll 1
    for (int t = blockIdx.y; t < T; t += gridDim.y)
        rows[(long long)t * H + r] = reduce_group(x + (long long)t * ldx + c0, 1, n, mode);
}

// reduce_group on values held in registers (n known at compile time)
__device__ __forceinline__ float reduce_vals(const float *v, int n, int mode) {
    if (mode == FILARK_VIEW_DROP || n == 1) return v[0];
    if (mode == FILARK_VIEW_PEAK) {
        float best = v[0], mag = fabsf(v[0]);
        for (int i = 1; i < n; ++i)
            if (fabsf(v[i]) > mag) {
                mag = fabsf(v[i]);
                best = v[i];
            }
        return best;
    }
    const int i0 = (n - 1) >> 1;
    if (n & 1) return v[i0];
    return 0.5f * v[i0] + 0.5f * v[i0 + 1];
}

// The same with G rows per thread read as 16-byte vectors (G * KC a multiple
// of 4, KC <= 8 channels per row known at compile time), rows of x 16-byte
// aligned; threads at the array's end take the scalar path.
template <int KC>
__host__ __device__ constexpr int rows_per_thread() {
    return KC % 4 == 0 ? 1 : (KC % 2 == 0 ? 2 : 4);
}

template <int KC>
__global__ void view_rows_vec_kernel(const float *__restrict__ x, long long ldx, int t0, int C, int H, int mode,
                                     float *__restrict__ rows) {
    constexpr int G = rows_per_thread<KC>(), NF = G * KC;
    const int ng = (H + G - 1) / G;
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;     // group of G rows
    if (gi >= ng) return;
    const int r0 = gi * G, c0 = r0 * KC;
    const int t = t0 + blockIdx.y;     // grid (groups of 256 x G rows, samples from t0)
    const float *xr = x + (long long)t * ldx;
    if (c0 + NF <= C && r0 + G <= H) {
        float v[NF];
#pragma unroll
        for (int q = 0; q < NF / 4; ++q) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(xr + c0) + q);
            v[4 * q] = f.x;
            v[4 * q + 1] = f.y;
            v[4 * q + 2] = f.z;
            v[4 * q + 3] = f.w;
        }
#pragma unroll
        for (int rr = 0; rr < G; ++rr) rows[(long long)t * H + r0 + rr] = reduce_vals(v + rr * KC, KC, mode);
    } else {
        for (int r = r0; r < min(H, r0 + G); ++r) {
            const int c = r * KC, n = min(C, c + KC) - c;
            rows[(long long)t * H + r] = reduce_group(xr + c, 1, n, mode);
        }
    }
}

template <int KC>
void launch_rows_vec(const float *x, long long ldx, int T, int C, int H, int mode, float *rows, cudaStream_t s) {
    const int ng = (H + rows_per_thread<KC>() - 1) / rows_per_thread<KC>();
    for (int t0 = 0; t0 < T; t0 += 65535) {
        const dim3 grid((unsigned)((ng + 255) / 256), (unsigned)std::min(T - t0, 65535));
        view_rows_vec_kernel<KC><<<grid, 256, 0, s>>>(x, ldx, t0, C, H, mode, rows);
    }
}

// Column q of this push covers virtual samples q*kt .. q*kt + kt - 1, where
// virtual sample v < nc is carry[v] and later ones are src[v - nc].
__device__ __forceinline__ float vsample(const float *carry, const float *src, int nc, int H, long long v, int r) {
    return v < nc ? carry[v * H + r] : src[(v - nc) * H + r];
}

// grid (row groups of 256, new columns): new column qi = blockIdx.y of the
// columns q0, q0 + 1, ... goes to ring column colq0 + qi (colq0 < W, qi < W)
__global__ void view_columns_kernel(const float *__restrict__ carry, const float *__restrict__ src, int nc,
                                    int H, int kt, int mode, long long q0, int colq0, int W,
                                    float *__restrict__ ring) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    const int qi = blockIdx.y;
    const long long v0 = (q0 + qi) * kt;
    float out;
    if (mode == FILARK_VIEW_DROP || kt == 1) {
        out = vsample(carry, src, nc, H, v0, r);
    } else if (mode == FILARK_VIEW_PEAK) {
        out = vsample(carry, src, nc, H, v0, r);
        float mag = fabsf(out);
        int k = 1;
        // four loads in flight, then the comparisons in order (first on ties)
        for (; k + 4 <= kt; k += 4) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = vsample(carry, src, nc, H, v0 + k + u, r);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (fabsf(v[u]) > mag) {
                    mag = fabsf(v[u]);
                    out = v[u];
                }
        }
        for (; k < kt; ++k) {
            const float v = vsample(carry, src, nc, H, v0 + k, r);
            if (fabsf(v) > mag) {
                mag = fabsf(v);
                out = v;
            }
        }
    } else {
        const int i0 = (kt - 1) >> 1;
        const float a = vsample(carry, src, nc, H, v0 + i0, r);
        out = (kt & 1) ? a : 0.5f * a + 0.5f * vsample(carry, src, nc, H, v0 + i0 + 1, r);
    }
    int col = colq0 + qi;
    if (col >= W) col -= W;
    ring[(long long)r * W + col] = out;
}

// new carry = virtual samples [from, from + n)
__global__ void view_carry_kernel(const float *__restrict__ carry, const float *__restrict__ src, int nc, int H,
                                  long long from, int n, float *__restrict__ carry_next) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * H) return;
    const int k = i / H, r = i % H;
    carry_next[i] = vsample(carry, src, nc, H, from + k, r);
}

// grid (image column groups of 256, rows; rows past gridDim.y loop); ncmod =
// ncols mod W
__global__ void view_image_kernel(const float *__restrict__ ring, int H, int W, long long ncols, int ncmod,
                                  float *__restrict__ img, long long ldi) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= W) return;
    const bool shown = ncols - W + c >= 0;    // global column ncols - W + c exists
    int j = ncmod + c;                        // its ring column, (ncols - W + c) mod W
    if (j >= W) j -= W;
#pragma unroll 1
    for (int r = blockIdx.y; r < H; r += gridDim.y)
        img[(long long)r * ldi + c] = shown ? ring[(long long)r * W + j] : 0.f;
}




unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

struct filark_view {
    int device = 0, C = 0, kc = 1, kt = 1, W = 1, H = 1, mode = 0;
    long long max_chunk = 0, n = 0, ncols = 0;
    filark_chain *filt = nullptr;
    float *rows = nullptr, *frows = nullptr;
    float *carry[2] = {nullptr, nullptr};
    int carry_n = 0, parity = 0;
    float *ring = nullptr;
};

namespace {

void free_view(filark_view *v) {
    if (!v) return;
    if (v->filt) filark_chain_destroy(v->filt);
    for (float *p : {v->rows, v->frows, v->carry[0], v->carry[1], v->ring})
        if (p) cudaFree(p);
    delete v;
}

}  // namespace

extern "C" {

filark_status filark_view_create(int n_channels, int channels_per_row, int samples_per_column, int width, int mode,
                                 int n_sections, const double *sos, int64_t max_chunk, int cuda_device,
                                 filark_view **out) {
    if (!out) return fail_with(FILARK_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_channels < 1 || channels_per_row < 1 || samples_per_column < 1 || width < 1 || max_chunk < 1)
        return fail_with(FILARK_EINVAL, "sizes must be >= 1");
    if (mode < FILARK_VIEW_DROP || mode > FILARK_VIEW_LINEAR) return fail_with(FILARK_EINVAL, "unknown view mode");
    if (n_sections < 0 || (n_sections > 0 && !sos)) return fail_with(FILARK_EINVAL, "display filter sections");
    filark_view *v = new (std::nothrow) filark_view();
    if (!v) return fail_with(FILARK_ENOMEM, "host allocation failed");
    v->device = cuda_device;
    v->C = n_channels;
    v->kc = channels_per_row;
    v->kt = samples_per_column;
    v->W = width;
    v->H = (n_channels + channels_per_row - 1) / channels_per_row;
    v->mode = mode;
    v->max_chunk = max_chunk;
    if (n_sections > 0) {
        filark_chain_config cfg{};
        cfg.abi_version = FILARK_ABI_VERSION;
        cfg.n_channels = v->H;
        cfg.fs = 1.0;
        cfg.n_sections = n_sections;
        cfg.sos = sos;
        cfg.spatial_width = 1;
        cfg.outputs = FILARK_OUT_BANDPASS;
        cfg.precision = FILARK_PREC_AUTO;
        cfg.max_chunk = max_chunk;
        filark_status st = filark_chain_create(&cfg, cuda_device, &v->filt);
        if (st != FILARK_OK) {
            const std::string msg = std::string("display filter: ") + filark_last_error_string();
            delete v;
            return fail_with(st, msg);
        }
    }
    DeviceGuard dg(cuda_device);
    if (!dg.ok) {
        free_view(v);
        return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    }
    const size_t H = (size_t)v->H;
    cudaError_t e = cudaMalloc(&v->rows, sizeof(float) * (size_t)max_chunk * H);
    if (e == cudaSuccess && v->filt) e = cudaMalloc(&v->frows, sizeof(float) * (size_t)max_chunk * H);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc(&v->carry[k], sizeof(float) * (size_t)v->kt * H);
    if (e == cudaSuccess) e = cudaMalloc(&v->ring, sizeof(float) * (size_t)v->W * H);
    if (e == cudaSuccess) e = cudaMemset(v->ring, 0, sizeof(float) * (size_t)v->W * H);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_view(v);
        return fail_cuda_with(e, "view create");
    }
    *out = v;
    return FILARK_OK;
}

filark_status filark_view_push(filark_view *v, const float *d_in, int64_t ld_in, int64_t n_samples,
                               filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_view_push");
    if (!v) return fail_with(FILARK_EINVAL, "view is NULL");
    if (n_samples < 0 || n_samples > v->max_chunk) return fail_with(FILARK_EINVAL, "n_samples must be in [0, max_chunk]");
    if (n_samples == 0) return FILARK_OK;
    if (!d_in || ld_in < v->C) return fail_with(FILARK_EINVAL, "input NULL or ld < n_channels");
    DeviceGuard dg(v->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    const int T = (int)n_samples, H = v->H;
    if (ld_in % 4 == 0 && ((uintptr_t)d_in & 15u) == 0 && v->kc <= 8) {
        switch (v->kc) {
        case 1: launch_rows_vec<1>(d_in, ld_in, T, v->C, H, v->mode, v->rows, s); break;
        case 2: launch_rows_vec<2>(d_in, ld_in, T, v->C, H, v->mode, v->rows, s); break;
        case 3: launch_rows_vec<3>(d_in, ld_in, T, v->C, H, v->mode, v->rows, s); break;
        case 4: launch_rows_vec<4>(d_in, ld_in, T, v->C, H, v->mode, v->rows, s); break;
        case 5: launch_rows_vec<5>(d_in, ld_in, T, v->C, H, v->mode, v->rows, s); break;
        case 6: launch_rows_vec<6>(d_in, ld_in, T, v->C, H, v->mode, v->rows, s); break;
        case 7: launch_rows_vec<7>(d_in, ld_in, T, v->C, H, v->mode, v->rows, s); break;
        default: launch_rows_vec<8>(d_in, ld_in, T, v->C, H, v->mode, v->rows, s); break;
        }
    } else {
        const dim3 grid((unsigned)((H + 255) / 256), (unsigned)std::min(T, 65535));
        view_rows_kernel<<<grid, 256, 0, s>>>(d_in, ld_in, T, v->C, v->kc, H, v->mode, v->rows);
    }
    const float *src = v->rows;
    if (v->filt) {
        filark_status st = filark_chain_push_chunk(v->filt, v->rows, H, T, nullptr, v->frows, nullptr, H, stream);
        if (st != FILARK_OK) return st;
        src = v->frows;
    }
    const long long avail = (long long)v->carry_n + T;
    const long long nq = avail / v->kt;
    // only the last W new columns survive in the ring
    const long long q0 = nq > v->W ? nq - v->W : 0;
    // new columns q0 .. nq - 1 (at most W), up to 65535 per launch
    for (long long qa = q0; qa < nq; qa += 65535) {
        const int nnew = (int)std::min<long long>(nq - qa, 65535);
        const int colq0 = (int)((v->ncols + qa) % v->W);
        const dim3 grid((unsigned)((H + 255) / 256), (unsigned)nnew);
        view_columns_kernel<<<grid, 256, 0, s>>>(v->carry[v->parity], src, v->carry_n, H, v->kt, v->mode, qa, colq0,
                                                 v->W, v->ring);
    }
    const int nrest = (int)(avail - nq * v->kt);
    if (nrest > 0)
        view_carry_kernel<<<blocks_for((long long)nrest * H), 256, 0, s>>>(v->carry[v->parity], src, v->carry_n, H,
                                                                           nq * v->kt, nrest,
                                                                           v->carry[v->parity ^ 1]);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda_with(e, "view push");
    v->parity ^= 1;
    v->carry_n = nrest;
    v->ncols += nq;
    v->n += T;
    return FILARK_OK;
}

filark_status filark_view_image(const filark_view *v, float *d_image, int64_t ld_image, filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_view_image");
    if (!v) return fail_with(FILARK_EINVAL, "view is NULL");
    if (!d_image || ld_image < v->W) return fail_with(FILARK_EINVAL, "image NULL or ld < width");
    DeviceGuard dg(v->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    const dim3 grid((unsigned)((v->W + 255) / 256), (unsigned)std::min(v->H, 65535));
    view_image_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(v->ring, v->H, v->W, v->ncols, (int)(v->ncols % v->W),
                                                              d_image, ld_image);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FILARK_OK : fail_cuda_with(e, "view image");
}

filark_status filark_view_get_info(const filark_view *v, int *rows, int64_t *columns, int *ring_offset) {
    if (!v) return fail_with(FILARK_EINVAL, "view is NULL");
    if (rows) *rows = v->H;
    if (columns) *columns = v->ncols;
    if (ring_offset) *ring_offset = (int)(v->ncols % v->W);
    return FILARK_OK;
}

filark_status filark_view_reset(filark_view *v, filark_stream_t stream) {
    if (!v) return fail_with(FILARK_EINVAL, "view is NULL");
    DeviceGuard dg(v->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    if (v->filt) {
        filark_status st = filark_chain_reset_state(v->filt, stream);
        if (st != FILARK_OK) return st;
    }
    const cudaError_t e = cudaMemsetAsync(v->ring, 0, sizeof(float) * (size_t)v->W * v->H, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda_with(e, "view reset");
    v->n = v->ncols = 0;
    v->carry_n = 0;
    return FILARK_OK;
}

filark_status filark_view_destroy(filark_view *v) {
    if (!v) return FILARK_OK;
    DeviceGuard dg(v->device);
    cudaDeviceSynchronize();
    free_view(v);
    return FILARK_OK;
}

}  // extern "C"
