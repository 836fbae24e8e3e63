// Allocation-free entry point: filark_chain_run_static (see include/filark.h).
//
// Some callers cannot call cudaMalloc: a real-time acquisition thread whose
// latency budget rules out an allocator call (cudaMalloc can block and
// synchronise), or a plugin inside a host application that owns all device
// memory through its own pool.  This entry point runs the whole chain over
// one recording, from a zero state, with the chain's working memory (carried
// IIR and detector state, cf history ring, dense-carry matrices) placed in a
// file-scope device array instead of cudaMalloc'd buffers.
//
// The array is kStaticScratchBytes (32 MiB); every GPU that loads the library
// holds it until the process exits.  All calls share it: each call clears what
// must start at zero, and calls that overlap on the GPU (different streams,
// or different host threads) race on it.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "filark_internal.h"

namespace filark {
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;

bool ranges_overlap(const void *a, size_t an, const void *b, size_t bn) {
    const char *pa = (const char *)a, *pb = (const char *)b;
    return pa < pb + bn && pb < pa + an;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

// Set the thread's error message shown by filark_last_error_string (api.cpp).
void set_last_error(const std::string &msg);

}  // namespace filark

using namespace filark;

extern "C" filark_status filark_chain_run_static(const filark_chain_config *cfg, const float *d_in,
                                                 int64_t ld_in, int64_t n_samples, float *d_ratio,
                                                 float *d_bandpass, float *d_spatial, int64_t ld_out,
                                                 filark_stream_t stream) {
    auto fail = [](filark_status st, const std::string &m) {
        set_last_error(m);
        return st;
    };
    if (!cfg) return fail(FILARK_EINVAL, "config is NULL");
    if (cfg->abi_version != FILARK_ABI_VERSION) return fail(FILARK_EINVAL, "abi_version mismatch");
    const int C = cfg->n_channels;
    if (C < 1) return fail(FILARK_EINVAL, "n_channels must be >= 1");
    if (!(cfg->fs > 0)) return fail(FILARK_EINVAL, "fs must be > 0");
    if (cfg->n_sections < 0) return fail(FILARK_EINVAL, "n_sections must be >= 0");
    if (cfg->n_sections > FILARK_MAX_SECTIONS) return fail(FILARK_ENOSYS, "more than FILARK_MAX_SECTIONS sections");
    if (cfg->n_sections > 0 && !cfg->sos) return fail(FILARK_EINVAL, "sos is NULL");
    if (cfg->spatial_width < 1 || cfg->spatial_width % 2 == 0)
        return fail(FILARK_EINVAL, "spatial_width must be odd and >= 1");
    if (cfg->spatial_width > FILARK_MAX_SPATIAL_WIDTH)
        return fail(FILARK_ENOSYS, "spatial_width above FILARK_MAX_SPATIAL_WIDTH");
    const bool det = cfg->lta_len > 0 || cfg->sta_len > 0;
    if (det && (cfg->sta_len < 1 || cfg->lta_len < cfg->sta_len))
        return fail(FILARK_EINVAL, "need 1 <= sta_len <= lta_len (or both 0)");
    if (n_samples < 0) return fail(FILARK_EINVAL, "n_samples must be >= 0");
    if (n_samples > 0 && !d_in) return fail(FILARK_EINVAL, "input is NULL");
    if (ld_in < C) return fail(FILARK_EINVAL, "ld_in < n_channels");
    if ((d_ratio || d_bandpass || d_spatial) && ld_out < C) return fail(FILARK_EINVAL, "ld_out < n_channels");
    if (d_ratio && !det) return fail(FILARK_EINVAL, "ratio output needs the detector");
    if (d_ratio && !(cfg->outputs & FILARK_OUT_RATIO)) return fail(FILARK_EINVAL, "ratio output not enabled");
    if (d_bandpass && !(cfg->outputs & FILARK_OUT_BANDPASS))
        return fail(FILARK_EINVAL, "bandpass output not enabled");
    if (d_spatial && !(cfg->outputs & FILARK_OUT_SPATIAL)) return fail(FILARK_EINVAL, "spatial output not enabled");
    if (n_samples > 0) {
        const size_t in_bytes = sizeof(float) * (size_t)((n_samples - 1) * ld_in + C);
        const size_t out_bytes = sizeof(float) * (size_t)((n_samples - 1) * std::max<int64_t>(ld_out, 0) + C);
        const void *outs[3] = {d_ratio, d_bandpass, d_spatial};
        for (int a = 0; a < 3; ++a) {
            if (outs[a] && ranges_overlap(d_in, in_bytes, outs[a], out_bytes))
                return fail(FILARK_EINVAL, "an output overlaps the input");
            for (int b = a + 1; b < 3; ++b)
                if (outs[a] && outs[b] && ranges_overlap(outs[a], out_bytes, outs[b], out_bytes))
                    return fail(FILARK_EINVAL, "two outputs overlap");
        }
    }
    if (cfg->precision < FILARK_PREC_AUTO || cfg->precision > FILARK_PREC_ALL32)
        return fail(FILARK_EINVAL, "unknown precision mode");

    Plan plan;
    std::string err;
    filark_status st = make_plan(cfg->sos, cfg->n_sections, cfg->precision, &plan, &err);
    if (st != FILARK_OK) return fail(st, err);
    const int NS = plan.NS;
    const int hw = (cfg->spatial_width - 1) / 2;
    const int HP = (hw + 3) / 4 * 4;
    const int Wout = kWT - 2 * HP;
    const int n_tiles = (C + Wout - 1) / Wout;
    const long long ldr = (C + 3) / 4 * 4;
    const long long Q = det ? (long long)cfg->lta_len + std::min<int64_t>(std::max<int64_t>(n_samples, 1), kMaxLaunchSamples) : 1;

    // carve the scratch: IIR state x2, detector state x2, ring, dense matrices
    const size_t b_iir = align256(sizeof(double) * (size_t)C * (size_t)(2 * NS));
    const size_t b_det = align256(sizeof(double) * (size_t)C * 4);
    const size_t b_ring = det ? align256(sizeof(float) * (size_t)Q * (size_t)ldr) : 0;
    const size_t b_dense = plan.dense ? align256(sizeof(float) * plan.dense_mats.size()) : 0;
    const size_t need = 2 * b_iir + 2 * b_det + b_ring + b_dense;
    if (need > kStaticScratchBytes || (double)Q * (double)ldr >= 2147483647.0)
        return fail(FILARK_EINVAL, "recording needs " + std::to_string(need) + " bytes of working memory; the static "
                    "array holds " + std::to_string(kStaticScratchBytes) + " (lower n_channels or lta_len)");
    if (n_samples == 0) return FILARK_OK;

    // The array's device address and the kernels' attributes are taken on
    // every call, on the current device: a cached address would outlive a
    // cudaDeviceReset (the module, and the array with it, is loaded again in
    // the new context).  Neither call allocates.
    char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return fail(FILARK_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        }
        e = configure_chain_kernels();
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(FILARK_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
        }
        base = (char *)ptr;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *iir[2] = {(double *)base, (double *)(base + b_iir)};
    double *dst[2] = {(double *)(base + 2 * b_iir), (double *)(base + 2 * b_iir + b_det)};
    float *ring = det ? (float *)(base + 2 * b_iir + 2 * b_det) : nullptr;
    float *dense = plan.dense ? (float *)(base + 2 * b_iir + 2 * b_det + b_ring) : nullptr;
    // zero state (the ring needs no clearing: every value read was written
    // earlier in this call, or lies before the first sample and reads as 0)
    cudaError_t e = cudaMemsetAsync(base, 0, 2 * b_iir + 2 * b_det, s);
    if (e == cudaSuccess && dense)
        e = cudaMemcpyAsync(dense, plan.dense_mats.data(), sizeof(float) * plan.dense_mats.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && dense) e = cudaStreamSynchronize(s);   // the host copy source is pageable
    if (e != cudaSuccess) return fail(FILARK_ECUDA, std::string("scratch clear: ") + cudaGetErrorString(e));

    ChainParams p;
    set_static_params(plan, hw, HP, Wout, cfg->sta_len, cfg->lta_len, dense, p);
    p.pdl = 1;
    ChainUnit &u = p.u;
    u.ring = ring;
    u.ldr = ldr;
    u.Q = (int)Q;
    u.C = C;
    int parity = 0;
    for (int64_t done = 0; done < n_samples;) {
        const int Tl = (int)std::min<int64_t>(n_samples - done, kMaxLaunchSamples);
        u.x = d_in + done * ld_in;
        u.ldx = ld_in;
        u.ratio = d_ratio ? d_ratio + done * ld_out : nullptr;
        u.bp = d_bandpass ? d_bandpass + done * ld_out : nullptr;
        u.sp = d_spatial ? d_spatial + done * ld_out : nullptr;
        u.ldo = ld_out;
        u.iir_in = iir[parity];
        u.iir_out = iir[parity ^ 1];
        u.det_in = dst[parity];
        u.det_out = dst[parity ^ 1];
        u.n0 = done;
        set_unit_geometry(plan, Tl, kNB, u);
        u.slot_n0 = (int)(done % Q);
        u.x_vec4 = (ld_in % 4 == 0) && (((uintptr_t)u.x & 15u) == 0);
        bool ov = (ld_out % 4 == 0);
        for (float *o : {u.ratio, u.bp, u.sp})
            if (o && ((uintptr_t)o & 15u)) ov = false;
        u.o_vec4 = ov;
        e = launch_chain(p, NS, det, plan.dense, n_tiles, s);
        if (e != cudaSuccess) return fail(FILARK_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
        parity ^= 1;
        done += Tl;
    }
    return FILARK_OK;
}
