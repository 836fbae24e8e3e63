// C-ABI of the chunked DAS filter chain (see include/filark.h).
//
// Owns the chain's device state and drives the fused kernel.  Every push is
// split into launches of at most kMaxLaunchSamples samples; each launch reads
// the carried state from one of two buffers and writes the next state to the
// other (the halo channels of a tile read a neighbour's state while that
// neighbour writes its own), so consecutive launches simply alternate.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "chain_object.h"
#include "host_trace.h"

using namespace filark;

namespace {

thread_local std::string g_err;

filark_status fail(filark_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

filark_status fail_cuda(cudaError_t e, const char *what) {
    cudaGetLastError();
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return FILARK_ECUDA;
}


std::mutex g_cfg_mu;

constexpr uint32_t kStateMagic = 0x4B524C46u;   // "FLRK"
constexpr uint32_t kStateVersion = 1u;

struct StateHeader {
    uint32_t magic, version;
    int32_t C, S, ns, nl, K, reserved;
    int64_t n;
    int64_t hist_rows;
};

}  // namespace

namespace filark {
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace filark

namespace {

void free_chain(filark_chain *h) {
    if (!h) return;
    for (int i = 0; i < 2; ++i) {
        if (h->iir[i]) cudaFree(h->iir[i]);
        if (h->detst[i]) cudaFree(h->detst[i]);
    }
    if (h->ring) cudaFree(h->ring);
    if (h->dense) cudaFree(h->dense);
    if (h->status_host) cudaFreeHost(h->status_host);
    for (float *p : h->stage)
        if (p) cudaFree(p);
    for (int k = 0; k < FILARK_HOST_SLOTS; ++k) {
        for (float *p : h->astage[k])
            if (p) cudaFree(p);
        if (h->ev_in[k]) cudaEventDestroy(h->ev_in[k]);
        if (h->ev_comp[k]) cudaEventDestroy(h->ev_comp[k]);
        if (h->ev_out[k]) cudaEventDestroy(h->ev_out[k]);
    }
    if (h->hcopy_in) cudaStreamDestroy(h->hcopy_in);
    if (h->hcopy_out) cudaStreamDestroy(h->hcopy_out);
    for (int l = 0; l < FILARK_MAX_LANES; ++l) {
        if (h->lane_s[l]) cudaStreamDestroy(h->lane_s[l]);
        if (h->ev_lane[l]) cudaEventDestroy(h->ev_lane[l]);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    for (double *p : h->halo)
        if (p) cudaFree(p);
    delete h;
}

bool ranges_overlap(const void *a, size_t an, const void *b, size_t bn) {
    const char *pa = (const char *)a, *pb = (const char *)b;
    return pa < pb + bn && pb < pa + an;
}

filark_status zero_state(filark_chain *h, cudaStream_t stream) {
    const int NS = h->plan.NS;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        if (h->iir[i]) e = cudaMemsetAsync(h->iir[i], 0, sizeof(double) * (size_t)h->C * (size_t)(2 * NS), stream);
        if (e == cudaSuccess && h->detst[i]) e = cudaMemsetAsync(h->detst[i], 0, sizeof(double) * (size_t)h->C * 4, stream);
    }
    if (e == cudaSuccess && h->ring)
        e = cudaMemsetAsync(h->ring, 0, sizeof(float) * (size_t)h->Q * (size_t)h->ldr, stream);
    if (e != cudaSuccess) return fail_cuda(e, "reset: cudaMemsetAsync");
    *(volatile int *)h->status_host = 0;
    h->parity = 0;
    h->n = 0;
    h->sticky = FILARK_OK;
    h->halo_valid = false;
    return FILARK_OK;
}

// The modal carries keep each state entry as a double-float {hi, lo} pair of
// floats in its 8-byte slot; the checkpoint format is FP64.
void decode_df_state(std::vector<double> &m) {
    for (double &v : m) {
        float hl[2];
        std::memcpy(hl, &v, sizeof(hl));
        v = (double)hl[0] + (double)hl[1];
    }
}

void encode_df_state(std::vector<double> &m) {
    for (double &v : m) {
        float hl[2];
        hl[0] = (float)v;
        hl[1] = (float)(v - (double)hl[0]);
        std::memcpy(&v, hl, sizeof(hl));
    }
}

filark_status check_device_status(filark_chain *h) {
    if (h->sticky != FILARK_OK) return fail(FILARK_ESTATE, "chain is in an error state; call filark_chain_reset_state");
    int st = *(volatile int *)h->status_host;
    if (st != 0) {
        h->sticky = FILARK_ETIMEOUT;
        return fail(FILARK_ESTATE, "a device-side error was reported (code " + std::to_string(st) + "); reset the chain");
    }
    return FILARK_OK;
}

// Make `stream` wait for every lane's enqueued work.
filark_status join_lanes(filark_chain *h, cudaStream_t stream) {
    if (!h->lanes_pending) return FILARK_OK;
    for (int l = 0; l < FILARK_MAX_LANES; ++l) {
        if (!h->lane_s[l]) continue;
        cudaError_t e = cudaEventRecord(h->ev_lane[l], h->lane_s[l]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, h->ev_lane[l], 0);
        if (e != cudaSuccess) {
            h->sticky = FILARK_ECUDA;
            return fail_cuda(e, "join: event");
        }
    }
    h->lanes_pending = false;
    return FILARK_OK;
}

// Enqueue one push.  With lanes, every launch of the push runs each tile group
// on its lane stream after the work already on `stream`; join_after makes
// `stream` wait for the lanes at the end (the host-buffer paths need their
// outputs on `stream`).
//
// Lane launches read only per-tile state (`halo`), which a tile alone writes.
// Until that state exists (after create, reset, set_state, a one-lane push or
// a lane change) a tile's halo columns would have to come from the
// neighbouring tiles' per-channel state, which another lane may already be
// overwriting; so the first launch in that case runs every tile at once on
// `stream` and writes the per-tile state, and the lanes fork after it.
filark_status push_device(filark_chain *h, const float *d_in, int64_t ld_in, int64_t T, float *d_ratio,
                          float *d_bp, float *d_sp, int64_t ld_out, cudaStream_t stream, bool join_after = false,
                          const TriggerFusion *tf = nullptr) {
    const int NS = h->plan.NS;
    const int L = std::min(h->lanes, h->n_tiles);
    bool forked = false;
    auto fork_lanes = [&]() -> filark_status {
        cudaError_t e = cudaEventRecord(h->ev_fork, stream);
        for (int l = 0; l < L && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(h->lane_s[l], h->ev_fork, 0);
        if (e != cudaSuccess) {
            h->sticky = FILARK_ECUDA;
            return fail_cuda(e, "push: lane fork");
        }
        forked = true;
        return FILARK_OK;
    };
    if (L <= 1 || !h->halo_valid) {
        filark_status st = join_lanes(h, stream);
        if (st != FILARK_OK) return st;
    }
    int64_t done = 0;
    while (done < T) {
        const int Tl = (int)std::min<int64_t>(T - done, h->launch_samples);
        ChainParams p = h->base;
        ChainUnit &u = p.u;
        u.x = d_in + done * ld_in;
        u.ldx = ld_in;
        u.ratio = d_ratio ? d_ratio + done * ld_out : nullptr;
        u.bp = d_bp ? d_bp + done * ld_out : nullptr;
        u.sp = d_sp ? d_sp + done * ld_out : nullptr;
        u.ldo = ld_out;
        u.iir_in = h->iir[h->parity];
        u.iir_out = h->iir[h->parity ^ 1];
        u.det_in = h->detst[h->parity];
        u.det_out = h->detst[h->parity ^ 1];
        u.n0 = h->n;
        // blocks per CTA: kNB unless the caller set fewer (the modal carry's
        // cross-CTA powers are tabulated per setting; the dense carry keeps kNB)
        const int nblk = (Tl + kL - 1) / kL;
        int nbc = kNB;
        if (!h->plan.dense && h->nbc_fixed > 0)
            nbc = std::max(h->nbc_fixed, (nblk + kMaxCluster - 1) / kMaxCluster);
        set_unit_geometry(h->plan, Tl, nbc, u);
        if (nbc != kNB) set_cta_powers(h->plan, nbc, p);
        u.slot_n0 = h->Q > 0 ? (int)(h->n % h->Q) : 0;
        p.pdl = h->use_pdl;
        u.x_vec4 = (ld_in % 4 == 0) && (((uintptr_t)u.x & 15u) == 0);
        bool ov = (ld_out % 4 == 0);
        for (float *o : {u.ratio, u.bp, u.sp})
            if (o && ((uintptr_t)o & 15u)) ov = false;
        u.o_vec4 = ov;
        // fused trigger summaries: the launch's blocks start at push block done / 32
        u.trig_summ = tf ? tf->summ + (size_t)(done / kL) * (size_t)h->C : nullptr;
        if (tf) {
            p.trig_on = tf->on;
            p.trig_off = tf->off;
        }
        auto launch = [&](int n_tiles, cudaStream_t q) {
            return tf ? launch_chain_trig(p, NS, h->plan.dense, n_tiles, q)
                      : launch_chain(p, NS, h->det, h->plan.dense, n_tiles, q);
        };
        cudaError_t e = cudaSuccess;
        if (L > 1 && !h->halo_valid) {
            // every tile in one launch on the caller's stream: halo columns
            // from the per-channel state, per-tile state written for the lanes
            u.halo_in = nullptr;
            u.halo_out = h->halo[h->parity ^ 1];
            u.tx0 = 0;
            e = launch(h->n_tiles, stream);
            h->halo_valid = true;
        } else if (L > 1) {
            if (!forked) {
                const filark_status st = fork_lanes();
                if (st != FILARK_OK) return st;
            }
            // each group reads and writes the state of its own tiles' columns
            u.halo_in = h->halo[h->parity];
            u.halo_out = h->halo[h->parity ^ 1];
            for (int l = 0; l < L && e == cudaSuccess; ++l) {
                const int t0 = (int)((long long)h->n_tiles * l / L), t1 = (int)((long long)h->n_tiles * (l + 1) / L);
                u.tx0 = t0;
                e = launch(t1 - t0, h->lane_s[l]);
            }
            h->lanes_pending = true;
        } else {
            e = launch(h->n_tiles, stream);
            h->halo_valid = false;
        }
        if (e != cudaSuccess) {
            h->sticky = FILARK_ECUDA;
            return fail_cuda(e, "push: kernel launch");
        }
        h->parity ^= 1;
        h->n += Tl;
        done += Tl;
    }
    if (join_after) return join_lanes(h, stream);
    return FILARK_OK;
}

filark_status validate_push(filark_chain *h, const void *in, int64_t ld_in, int64_t T, const void *ratio,
                            const void *bp, const void *sp, int64_t ld_out) {
    if (!h) return fail(FILARK_EINVAL, "chain is NULL");
    if (T < 0 || T > h->cfg.max_chunk) return fail(FILARK_EINVAL, "n_samples must be in [0, max_chunk]");
    if (T == 0) return FILARK_OK;
    if (!in) return fail(FILARK_EINVAL, "input is NULL");
    if (ld_in < h->C) return fail(FILARK_EINVAL, "ld_in < n_channels");
    const bool any_out = ratio || bp || sp;
    if (any_out && ld_out < h->C) return fail(FILARK_EINVAL, "ld_out < n_channels");
    if (ratio && (!(h->cfg.outputs & FILARK_OUT_RATIO) || !h->det))
        return fail(FILARK_EINVAL, "ratio output not enabled (outputs mask / detector off)");
    if (bp && !(h->cfg.outputs & FILARK_OUT_BANDPASS)) return fail(FILARK_EINVAL, "bandpass output not enabled");
    if (sp && !(h->cfg.outputs & FILARK_OUT_SPATIAL)) return fail(FILARK_EINVAL, "spatial output not enabled");
    const size_t in_bytes = sizeof(float) * (size_t)((T - 1) * ld_in + h->C);
    const size_t out_bytes = sizeof(float) * (size_t)((T - 1) * std::max<int64_t>(ld_out, 0) + h->C);
    for (const void *o : {ratio, bp, sp})
        if (o && ranges_overlap(in, in_bytes, o, out_bytes)) return fail(FILARK_EINVAL, "an output overlaps the input");
    const void *outs[3] = {ratio, bp, sp};
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (outs[a] && outs[b] && ranges_overlap(outs[a], out_bytes, outs[b], out_bytes))
                return fail(FILARK_EINVAL, "two outputs overlap");
    return FILARK_OK;
}

}  // namespace

namespace filark {
filark_status chain_zero_state(filark_chain *h, cudaStream_t stream) { return zero_state(h, stream); }
filark_status chain_check_status(filark_chain *h) { return check_device_status(h); }
filark_status chain_validate_push(filark_chain *h, const void *in, int64_t ld_in, int64_t T, const void *ratio,
                                  const void *bp, const void *sp, int64_t ld_out) {
    return validate_push(h, in, ld_in, T, ratio, bp, sp, ld_out);
}
}  // namespace filark

extern "C" {

uint32_t filark_abi_version(void) { return FILARK_ABI_VERSION; }

const char *filark_last_error_string(void) { return g_err.c_str(); }

filark_status filark_butter_bandpass_sos(int order, double f1, double f2, double fs, double *sos_out) {
    std::string err;
    filark_status st = design_butter_bandpass(order, f1, f2, fs, sos_out, &err);
    if (st != FILARK_OK) return fail(st, err);
    return FILARK_OK;
}

filark_status filark_chain_create(const filark_chain_config *cfg, int cuda_device, filark_chain **out) {
    if (!out) return fail(FILARK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(FILARK_EINVAL, "config is NULL");
    if (cfg->abi_version != FILARK_ABI_VERSION) return fail(FILARK_EINVAL, "abi_version mismatch");
    if (cfg->n_channels < 1) return fail(FILARK_EINVAL, "n_channels must be >= 1");
    if (!(cfg->fs > 0) || !std::isfinite(cfg->fs)) return fail(FILARK_EINVAL, "fs must be > 0");
    if (cfg->n_sections < 0) return fail(FILARK_EINVAL, "n_sections must be >= 0");
    if (cfg->n_sections > FILARK_MAX_SECTIONS)
        return fail(FILARK_ENOSYS, "more than FILARK_MAX_SECTIONS sections");
    if (cfg->n_sections > 0 && !cfg->sos) return fail(FILARK_EINVAL, "sos is NULL");
    if (cfg->spatial_width < 1 || cfg->spatial_width % 2 == 0)
        return fail(FILARK_EINVAL, "spatial_width must be odd and >= 1");
    if (cfg->spatial_width > FILARK_MAX_SPATIAL_WIDTH)
        return fail(FILARK_ENOSYS, "spatial_width above FILARK_MAX_SPATIAL_WIDTH");
    const bool det = cfg->lta_len > 0 || cfg->sta_len > 0;
    if (det && (cfg->sta_len < 1 || cfg->lta_len < cfg->sta_len))
        return fail(FILARK_EINVAL, "need 1 <= sta_len <= lta_len (or both 0)");
    if (cfg->sta_len < 0 || cfg->lta_len < 0) return fail(FILARK_EINVAL, "negative window length");
    if (cfg->outputs & ~(uint32_t)(FILARK_OUT_RATIO | FILARK_OUT_BANDPASS | FILARK_OUT_SPATIAL))
        return fail(FILARK_EINVAL, "unknown output bits");
    if ((cfg->outputs & FILARK_OUT_RATIO) && !det) return fail(FILARK_EINVAL, "ratio output needs the detector");
    if (cfg->max_chunk < 1) return fail(FILARK_EINVAL, "max_chunk must be >= 1");
    if (cfg->precision < FILARK_PREC_AUTO || cfg->precision > FILARK_PREC_ALL32)
        return fail(FILARK_EINVAL, "unknown precision mode");
    if (cfg->lta_len > (1 << 28)) return fail(FILARK_ENOSYS, "lta_len too large");

    filark_chain *h = new (std::nothrow) filark_chain();
    if (!h) return fail(FILARK_ENOMEM, "host allocation failed");
    h->cfg = *cfg;
    h->sos.assign(cfg->sos ? cfg->sos : (const double *)nullptr,
                  cfg->sos ? cfg->sos + 6 * cfg->n_sections : (const double *)nullptr);
    h->cfg.sos = h->sos.empty() ? nullptr : h->sos.data();
    std::string err;
    filark_status st = make_plan(h->sos.data(), cfg->n_sections, cfg->precision, &h->plan, &err);
    if (st != FILARK_OK) {
        delete h;
        return fail(st, err);
    }
    h->device = cuda_device;
    h->C = cfg->n_channels;
    h->K = cfg->spatial_width;
    h->hw = (h->K - 1) / 2;
    h->HP = (h->hw + 3) / 4 * 4;
    h->Wout = kWT - 2 * h->HP;
    h->n_tiles = (h->C + h->Wout - 1) / h->Wout;
    h->det = det;
    h->ns = cfg->sta_len;
    h->nl = cfg->lta_len;

    DeviceGuard dg(cuda_device);
    if (!dg.ok) {
        delete h;
        return fail(FILARK_ECUDA, "cudaSetDevice failed for device " + std::to_string(cuda_device));
    }
    {
        // set on every create: attributes set once would not survive a
        // cudaDeviceReset of the device
        std::lock_guard<std::mutex> lk(g_cfg_mu);
        cudaError_t e = configure_chain_kernels();
        if (e != cudaSuccess) {
            delete h;
            return fail_cuda(e, "create: kernel attributes");
        }
    }
    const int NS = h->plan.NS;
    auto alloc = [&](void **p, size_t bytes) -> bool {
        if (bytes == 0) return true;
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        h->device_bytes += (int64_t)bytes;
        return true;
    };
    bool ok = true;
    for (int i = 0; i < 2 && ok; ++i) {
        if (NS > 0) ok = ok && alloc((void **)&h->iir[i], sizeof(double) * (size_t)h->C * (size_t)(2 * NS));
        if (det) ok = ok && alloc((void **)&h->detst[i], sizeof(double) * (size_t)h->C * 4);
    }
    if (ok && det) {
        h->Q = (long long)h->nl + std::min<int64_t>(cfg->max_chunk, kMaxLaunchSamples);
        h->ldr = (h->C + 3) / 4 * 4;
        if ((double)h->Q * (double)h->ldr >= 2147483647.0) {
            free_chain(h);
            return fail(FILARK_ENOSYS, "detector history ring above 2^31 elements (lta_len x channels too large)");
        }
        ok = alloc((void **)&h->ring, sizeof(float) * (size_t)h->Q * (size_t)h->ldr);
    }
    if (ok && h->plan.dense) {
        ok = alloc((void **)&h->dense, sizeof(float) * h->plan.dense_mats.size());
        if (ok && cudaMemcpy(h->dense, h->plan.dense_mats.data(), sizeof(float) * h->plan.dense_mats.size(),
                             cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
        }
    }
    if (ok) {
        if (cudaHostAlloc((void **)&h->status_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer((void **)&h->status_dev, h->status_host, 0) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
        }
    }
    if (!ok) {
        free_chain(h);
        return fail(FILARK_ENOMEM, "device allocation failed");
    }
    // kernel parameter template
    ChainParams &b = h->base;
    set_static_params(h->plan, h->hw, h->HP, h->Wout, h->ns, h->nl, h->dense, b);
    b.u.ring = h->ring;
    b.u.ldr = h->ldr;
    b.u.Q = h->Q > 0 ? (int)h->Q : 1;
    b.u.C = h->C;
    b.u.nbc = kNB;

    st = zero_state(h, nullptr);
    if (st == FILARK_OK) {
        cudaError_t e = cudaStreamSynchronize(nullptr);
        if (e != cudaSuccess) st = fail_cuda(e, "create: synchronize");
    }
    if (st != FILARK_OK) {
        free_chain(h);
        return st;
    }
    *out = h;
    return FILARK_OK;
}

filark_status filark_chain_destroy(filark_chain *h) {
    if (!h) return FILARK_OK;
    DeviceGuard dg(h->device);
    cudaDeviceSynchronize();
    free_chain(h);
    return FILARK_OK;
}

filark_status filark_chain_reset_state(filark_chain *h, filark_stream_t stream) {
    if (!h) return fail(FILARK_EINVAL, "chain is NULL");
    DeviceGuard dg(h->device);
    const filark_status st = join_lanes(h, (cudaStream_t)stream);
    if (st != FILARK_OK) return st;
    return zero_state(h, (cudaStream_t)stream);
}

filark_status filark_chain_push_chunk(filark_chain *h, const float *d_in, int64_t ld_in, int64_t n_samples,
                                      float *d_ratio, float *d_bandpass, float *d_spatial, int64_t ld_out,
                                      filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_chain_push_chunk");
    filark_status st = validate_push(h, d_in, ld_in, n_samples, d_ratio, d_bandpass, d_spatial, ld_out);
    if (st != FILARK_OK) return st;
    st = check_device_status(h);
    if (st != FILARK_OK) return st;
    if (n_samples == 0) return FILARK_OK;
    DeviceGuard dg(h->device);
    return push_device(h, d_in, ld_in, n_samples, d_ratio, d_bandpass, d_spatial, ld_out, (cudaStream_t)stream);
}

filark_status filark_chain_push_triggers(filark_chain *h, filark_trigger *t, const float *d_in, int64_t ld_in,
                                        int64_t n_samples, float *d_ratio, int64_t ld_out,
                                        filark_trigger_record *d_records, int64_t capacity,
                                        unsigned long long *d_count, filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_chain_push_triggers");
    if (!t) return fail(FILARK_EINVAL, "trigger is NULL");
    if (!d_ratio) return fail(FILARK_EINVAL, "push_triggers needs the ratio output");
    filark_status st = validate_push(h, d_in, ld_in, n_samples, d_ratio, nullptr, nullptr, ld_out);
    if (st != FILARK_OK) return st;
    if (!d_count || capacity < 0 || (capacity > 0 && !d_records))
        return fail(FILARK_EINVAL, "records/capacity/count arguments");
    st = check_device_status(h);
    if (st != FILARK_OK) return st;
    if (n_samples == 0) return FILARK_OK;
    DeviceGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    TriggerFusion tf;
    st = trigger_fusion_begin(t, s, tf);
    if (st != FILARK_OK) return st;
    if (tf.C != h->C) return fail(FILARK_EINVAL, "trigger and chain have different channel counts");
    if (n_samples > tf.max_chunk) return fail(FILARK_EINVAL, "n_samples above the trigger's max_chunk");
    // The scan reads every tile's summaries: with the trigger on its own
    // stream it waits for this push's lane launches (the lanes go on with the
    // next push); otherwise the lanes join back into `stream`.
    const int L = std::min(h->lanes, h->n_tiles);
    const bool direct = tf.overlap && L > 1;
    st = push_device(h, d_in, ld_in, n_samples, d_ratio, nullptr, nullptr, ld_out, s, !direct, &tf);
    if (st != FILARK_OK) return st;
    cudaEvent_t deps[FILARK_MAX_LANES];
    int n_deps = 0;
    if (direct && h->lanes_pending) {
        for (int l = 0; l < L; ++l) {
            const cudaError_t e = cudaEventRecord(h->ev_lane[l], h->lane_s[l]);
            if (e != cudaSuccess) {
                h->sticky = FILARK_ECUDA;
                return fail_cuda(e, "push_triggers: lane event");
            }
            deps[n_deps++] = h->ev_lane[l];
        }
    }
    return trigger_push_summarized(t, d_ratio, ld_out, n_samples, d_records, capacity, d_count, s, deps, n_deps);
}

filark_status filark_chain_push_chunk_host(filark_chain *h, const float *h_in, int64_t ld_in, int64_t n_samples,
                                           float *h_ratio, float *h_bandpass, float *h_spatial, int64_t ld_out,
                                           filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_chain_push_chunk_host");
    filark_status st = validate_push(h, h_in, ld_in, n_samples, h_ratio, h_bandpass, h_spatial, ld_out);
    if (st != FILARK_OK) return st;
    st = check_device_status(h);
    if (st != FILARK_OK) return st;
    if (n_samples == 0) return FILARK_OK;
    DeviceGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t plane = sizeof(float) * (size_t)h->cfg.max_chunk * (size_t)h->C;
    float *hosts[4] = {const_cast<float *>(h_in), h_ratio, h_bandpass, h_spatial};
    for (int i = 0; i < 4; ++i) {
        if (hosts[i] && !h->stage[i]) {
            if (cudaMalloc((void **)&h->stage[i], plane) != cudaSuccess) {
                cudaGetLastError();
                return fail(FILARK_ENOMEM, "push_host: staging allocation failed");
            }
            h->device_bytes += (int64_t)plane;
        }
    }
    const size_t row = sizeof(float) * (size_t)h->C;
    cudaError_t e = cudaMemcpy2DAsync(h->stage[0], row, h_in, sizeof(float) * (size_t)ld_in, row,
                                      (size_t)n_samples, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_cuda(e, "push_host: input copy");
    st = push_device(h, h->stage[0], h->C, n_samples, h_ratio ? h->stage[1] : nullptr,
                     h_bandpass ? h->stage[2] : nullptr, h_spatial ? h->stage[3] : nullptr, h->C, s, true);
    if (st != FILARK_OK) return st;
    for (int i = 1; i < 4; ++i) {
        if (!hosts[i]) continue;
        e = cudaMemcpy2DAsync(hosts[i], sizeof(float) * (size_t)ld_out, h->stage[i], row, row, (size_t)n_samples,
                              cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return fail_cuda(e, "push_host: output copy");
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "push_host: synchronize");
    return check_device_status(h);
}

filark_status filark_chain_push_host_async(filark_chain *h, const float *h_in, int64_t ld_in, int64_t n_samples,
                                           float *h_ratio, float *h_bandpass, float *h_spatial, int64_t ld_out,
                                           filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_chain_push_host_async");
    filark_status st = validate_push(h, h_in, ld_in, n_samples, h_ratio, h_bandpass, h_spatial, ld_out);
    if (st != FILARK_OK) return st;
    st = check_device_status(h);
    if (st != FILARK_OK) return st;
    if (n_samples == 0) return FILARK_OK;
    DeviceGuard dg(h->device);
    cudaError_t e = cudaSuccess;
    if (!h->hcopy_in) {
        e = cudaStreamCreateWithFlags(&h->hcopy_in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->hcopy_out, cudaStreamNonBlocking);
        for (int k = 0; k < FILARK_HOST_SLOTS && e == cudaSuccess; ++k) {
            e = cudaEventCreateWithFlags(&h->ev_in[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_comp[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return fail_cuda(e, "push_host_async: stream/event creation");
    }
    const int k = h->aslot;
    const size_t plane = sizeof(float) * (size_t)h->cfg.max_chunk * (size_t)h->C;
    float *hosts[4] = {const_cast<float *>(h_in), h_ratio, h_bandpass, h_spatial};
    for (int i = 0; i < 4; ++i) {
        if (hosts[i] && !h->astage[k][i]) {
            if (cudaMalloc((void **)&h->astage[k][i], plane) != cudaSuccess) {
                cudaGetLastError();
                return fail(FILARK_ENOMEM, "push_host_async: staging allocation failed");
            }
            h->device_bytes += (int64_t)plane;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t row = sizeof(float) * (size_t)h->C;
    // input copy, once the slot's previous push has read its input
    if (h->slot_used[k]) e = cudaStreamWaitEvent(h->hcopy_in, h->ev_comp[k], 0);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(h->astage[k][0], row, h_in, sizeof(float) * (size_t)ld_in, row, (size_t)n_samples,
                              cudaMemcpyHostToDevice, h->hcopy_in);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[k], h->hcopy_in);
    // the push, once the input is in and the slot's previous outputs are out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_in[k], 0);
    if (e == cudaSuccess && h->slot_used[k]) e = cudaStreamWaitEvent(s, h->ev_out[k], 0);
    if (e != cudaSuccess) return fail_cuda(e, "push_host_async: input copy");
    st = push_device(h, h->astage[k][0], h->C, n_samples, h_ratio ? h->astage[k][1] : nullptr,
                     h_bandpass ? h->astage[k][2] : nullptr, h_spatial ? h->astage[k][3] : nullptr, h->C, s,
                     true);
    if (st != FILARK_OK) return st;
    e = cudaEventRecord(h->ev_comp[k], s);
    // output copies
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->hcopy_out, h->ev_comp[k], 0);
    for (int i = 1; i < 4 && e == cudaSuccess; ++i) {
        if (!hosts[i]) continue;
        e = cudaMemcpy2DAsync(hosts[i], sizeof(float) * (size_t)ld_out, h->astage[k][i], row, row, (size_t)n_samples,
                              cudaMemcpyDeviceToHost, h->hcopy_out);
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_out[k], h->hcopy_out);
    if (e != cudaSuccess) return fail_cuda(e, "push_host_async: output copy");
    h->slot_used[k] = true;
    h->aslot = (k + 1) % FILARK_HOST_SLOTS;
    return FILARK_OK;
}

filark_status filark_chain_host_sync(filark_chain *h, filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_chain_host_sync");
    if (!h) return fail(FILARK_EINVAL, "chain is NULL");
    DeviceGuard dg(h->device);
    const filark_status jst = join_lanes(h, (cudaStream_t)stream);
    if (jst != FILARK_OK) return jst;
    cudaError_t e = cudaSuccess;
    if (h->hcopy_in) e = cudaStreamSynchronize(h->hcopy_in);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess && h->hcopy_out) e = cudaStreamSynchronize(h->hcopy_out);
    if (e != cudaSuccess) {
        h->sticky = FILARK_ECUDA;
        return fail_cuda(e, "host_sync");
    }
    return check_device_status(h);
}

filark_status filark_chain_set_blocks_per_cta(filark_chain *h, int blocks_per_cta) {
    if (!h) return fail(FILARK_EINVAL, "chain is NULL");
    if (blocks_per_cta < 0 || blocks_per_cta > kNB) return fail(FILARK_EINVAL, "blocks_per_cta must be in 0..8");
    h->nbc_fixed = blocks_per_cta;
    return FILARK_OK;
}

filark_status filark_chain_set_launch_samples(filark_chain *h, int samples) {
    if (!h) return fail(FILARK_EINVAL, "chain is NULL");
    if (samples == 0) samples = kMaxLaunchSamples;
    if (samples < kTileRows || samples > kMaxLaunchSamples || samples % kTileRows != 0)
        return fail(FILARK_EINVAL, "samples per launch must be a multiple of 256 in 256..2048");
    h->launch_samples = samples;
    return FILARK_OK;
}

filark_status filark_chain_set_lanes(filark_chain *h, int lanes) {
    if (!h) return fail(FILARK_EINVAL, "chain is NULL");
    if (lanes < 1 || lanes > FILARK_MAX_LANES) return fail(FILARK_EINVAL, "lanes must be in 1..FILARK_MAX_LANES");
    DeviceGuard dg(h->device);
    // a tile may move to another lane: let the lanes' pending work finish
    for (int l = 0; l < FILARK_MAX_LANES && h->lanes_pending; ++l) {
        if (!h->lane_s[l]) continue;
        const cudaError_t e = cudaStreamSynchronize(h->lane_s[l]);
        if (e != cudaSuccess) {
            h->sticky = FILARK_ECUDA;
            return fail_cuda(e, "set_lanes: synchronize");
        }
    }
    h->lanes_pending = false;
    if (lanes > 1) {
        cudaError_t e = cudaSuccess;
        if (!h->ev_fork) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        for (int l = 0; l < lanes && e == cudaSuccess; ++l) {
            if (!h->lane_s[l]) e = cudaStreamCreateWithFlags(&h->lane_s[l], cudaStreamNonBlocking);
            if (e == cudaSuccess && !h->ev_lane[l]) e = cudaEventCreateWithFlags(&h->ev_lane[l], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return fail_cuda(e, "set_lanes: stream/event creation");
        const int NS = h->plan.NS;
        const size_t bytes = sizeof(double) * (size_t)h->n_tiles * kWT * (size_t)(2 * NS);
        for (int i = 0; i < 2 && bytes > 0; ++i) {
            if (h->halo[i]) continue;
            if (cudaMalloc((void **)&h->halo[i], bytes) != cudaSuccess) {
                cudaGetLastError();
                return fail(FILARK_ENOMEM, "set_lanes: halo state allocation failed");
            }
            h->device_bytes += (int64_t)bytes;
        }
    }
    h->lanes = lanes;
    return FILARK_OK;
}

filark_status filark_chain_tune(filark_chain *h, const float *d_in, int64_t ld_in, int64_t n_samples, float *d_ratio,
                                float *d_bandpass, float *d_spatial, int64_t ld_out, int timed_pushes,
                                filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_chain_tune");
    filark_status st = validate_push(h, d_in, ld_in, n_samples, d_ratio, d_bandpass, d_spatial, ld_out);
    if (st != FILARK_OK) return st;
    if (n_samples < 1 || timed_pushes < 1) return fail(FILARK_EINVAL, "tune needs n_samples >= 1 and timed_pushes >= 1");
    st = check_device_status(h);
    if (st != FILARK_OK) return st;
    DeviceGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e != cudaSuccess) {
        if (t0) cudaEventDestroy(t0);
        return fail_cuda(e, "tune: events");
    }
    // lanes x samples per launch x blocks per CTA (the dense carry keeps 8)
    struct Cand {
        int lanes, launch, blocks;
    };
    std::vector<Cand> cands;
    for (int blocks : {0, 4}) {
        if (blocks && h->plan.dense) continue;
        for (int launch : {kMaxLaunchSamples, kMaxLaunchSamples / 2})
            for (int lanes = 1; lanes <= std::min(FILARK_MAX_LANES, h->n_tiles); ++lanes)
                if ((int)cands.size() < 16) cands.push_back(Cand{lanes, launch, blocks});
    }
    h->n_tuned = 0;
    h->tuned_choice = -1;
    double best = 1e300;
    for (const Cand &c : cands) {
        st = filark_chain_set_lanes(h, c.lanes);
        if (st != FILARK_OK) break;
        h->launch_samples = c.launch;
        h->nbc_fixed = c.blocks;
        st = filark_chain_reset_state(h, stream);
        // two warm-up pushes, then timed_pushes back to back, joined at the end
        for (int w = 0; w < 2 && st == FILARK_OK; ++w)
            st = push_device(h, d_in, ld_in, n_samples, d_ratio, d_bandpass, d_spatial, ld_out, s);
        if (st == FILARK_OK && (e = cudaEventRecord(t0, s)) != cudaSuccess) st = fail_cuda(e, "tune: record");
        for (int q = 0; q < timed_pushes && st == FILARK_OK; ++q)
            st = push_device(h, d_in, ld_in, n_samples, d_ratio, d_bandpass, d_spatial, ld_out, s);
        if (st == FILARK_OK) st = join_lanes(h, s);
        if (st == FILARK_OK && (e = cudaEventRecord(t1, s)) != cudaSuccess) st = fail_cuda(e, "tune: record");
        if (st == FILARK_OK && (e = cudaEventSynchronize(t1)) != cudaSuccess) st = fail_cuda(e, "tune: sync");
        float ms = 0.f;
        if (st == FILARK_OK && (e = cudaEventElapsedTime(&ms, t0, t1)) != cudaSuccess)
            st = fail_cuda(e, "tune: elapsed");
        if (st != FILARK_OK) break;
        const double per = (double)ms / timed_pushes;
        const int k = h->n_tuned++;
        h->tune_lanes[k] = c.lanes;
        h->tune_launch[k] = c.launch;
        h->tune_blocks[k] = c.blocks;
        h->tune_ms[k] = per;
        if (per < best) {
            best = per;
            h->tuned_choice = k;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st != FILARK_OK) return st;
    const int k = h->tuned_choice;
    st = filark_chain_set_lanes(h, h->tune_lanes[k]);
    if (st != FILARK_OK) return st;
    h->launch_samples = h->tune_launch[k];
    h->nbc_fixed = h->tune_blocks[k];
    st = filark_chain_reset_state(h, stream);
    if (st == FILARK_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = fail_cuda(e, "tune: sync");
    return st;
}

filark_status filark_chain_get_tuning(const filark_chain *h, filark_chain_tuning *out) {
    if (!h || !out) return fail(FILARK_EINVAL, "chain or out is NULL");
    std::memset(out, 0, sizeof(*out));
    out->n_tuned = h->n_tuned;
    out->chosen = h->tuned_choice;
    for (int i = 0; i < h->n_tuned; ++i) {
        out->lanes[i] = h->tune_lanes[i];
        out->launch_samples[i] = h->tune_launch[i];
        out->blocks_per_cta[i] = h->tune_blocks[i];
        out->ms_per_push[i] = h->tune_ms[i];
    }
    return FILARK_OK;
}

filark_status filark_chain_join(filark_chain *h, filark_stream_t stream) {
    if (!h) return fail(FILARK_EINVAL, "chain is NULL");
    DeviceGuard dg(h->device);
    return join_lanes(h, (cudaStream_t)stream);
}

filark_status filark_chain_sync_status(filark_chain *h, filark_stream_t stream) {
    if (!h) return fail(FILARK_EINVAL, "chain is NULL");
    DeviceGuard dg(h->device);
    const filark_status jst = join_lanes(h, (cudaStream_t)stream);
    if (jst != FILARK_OK) return jst;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        h->sticky = FILARK_ECUDA;
        return fail_cuda(e, "sync_status");
    }
    return check_device_status(h);
}

filark_status filark_chain_get_info(const filark_chain *h, filark_chain_info *out) {
    if (!h || !out) return fail(FILARK_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->precision = h->plan.mode;
    out->block_len = kL;
    out->blocks_per_cta = kNB;
    out->tile_channels = h->Wout;
    out->halo = h->hw;
    out->n_slots = h->plan.NS;
    out->modal_condition = h->plan.kappa;
    out->probe_error = h->plan.probe_err;
    out->ring_len = h->Q;
    out->device_bytes = h->device_bytes;
    out->samples = h->n;
    return FILARK_OK;
}

filark_status filark_chain_get_state(filark_chain *h, void *host_buf, size_t *bytes, filark_stream_t stream) {
    if (!h || !bytes) return fail(FILARK_EINVAL, "NULL argument");
    const int S = h->plan.S, NS = h->plan.NS, C = h->C;
    const int64_t hist = h->det ? std::min<int64_t>(h->n, h->nl) : 0;
    const size_t need = sizeof(StateHeader) + sizeof(double) * (size_t)C * (size_t)(2 * S) +
                        sizeof(double) * (size_t)C * 3 + sizeof(float) * (size_t)hist * (size_t)C;
    if (!host_buf) {
        *bytes = need;
        return FILARK_OK;
    }
    if (*bytes < need) return fail(FILARK_EINVAL, "state buffer too small");
    DeviceGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    filark_status jst = join_lanes(h, s);
    if (jst != FILARK_OK) return jst;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "get_state: synchronize");
    filark_status st = check_device_status(h);
    if (st != FILARK_OK) return st;
    char *p = (char *)host_buf;
    StateHeader hd{kStateMagic, kStateVersion, C, S, h->ns, h->nl, h->K, 0, h->n, hist};
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    if (S > 0) {
        std::vector<double> m((size_t)C * (size_t)(2 * NS));
        e = cudaMemcpy(m.data(), h->iir[h->parity], sizeof(double) * m.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail_cuda(e, "get_state: copy");
        if (!h->plan.dense) decode_df_state(m);
        const int n2 = 2 * S;
        std::vector<double> canon((size_t)C * (size_t)n2);
        for (int c = 0; c < C; ++c)
            for (int r = 0; r < n2; ++r) {
                long double acc = 0;
                for (int q = 0; q < n2; ++q)
                    acc += h->plan.W[(size_t)r * n2 + q] * (long double)m[(size_t)c * (2 * NS) + q];
                canon[(size_t)c * n2 + r] = (double)acc;
            }
        std::memcpy(p, canon.data(), sizeof(double) * canon.size());
        p += sizeof(double) * canon.size();
    }
    std::vector<double> d((size_t)C * 4, 0.0);
    if (h->det) {
        e = cudaMemcpy(d.data(), h->detst[h->parity], sizeof(double) * d.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail_cuda(e, "get_state: copy");
    }
    for (int c = 0; c < C; ++c) std::memcpy(p + sizeof(double) * 3 * (size_t)c, &d[(size_t)c * 4], sizeof(double) * 3);
    p += sizeof(double) * 3 * (size_t)C;
    for (int64_t k = 0; k < hist; ++k) {
        const long long nabs = h->n - hist + k;
        const long long slot = nabs % h->Q;
        e = cudaMemcpy(p, h->ring + slot * h->ldr, sizeof(float) * (size_t)C, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail_cuda(e, "get_state: copy");
        p += sizeof(float) * (size_t)C;
    }
    *bytes = need;
    return FILARK_OK;
}

filark_status filark_chain_set_state(filark_chain *h, const void *host_buf, size_t bytes, filark_stream_t stream) {
    if (!h || !host_buf) return fail(FILARK_EINVAL, "NULL argument");
    if (bytes < sizeof(StateHeader)) return fail(FILARK_EINVAL, "state buffer too small");
    StateHeader hd;
    std::memcpy(&hd, host_buf, sizeof(hd));
    const int S = h->plan.S, NS = h->plan.NS, C = h->C;
    if (hd.magic != kStateMagic || hd.version != kStateVersion) return fail(FILARK_EINVAL, "not a filark state");
    if (hd.C != C || hd.S != S || hd.ns != h->ns || hd.nl != h->nl || hd.K != h->K || hd.n < 0)
        return fail(FILARK_EINVAL, "state does not match this chain's configuration");
    const int64_t hist = h->det ? std::min<int64_t>(hd.n, h->nl) : 0;
    if (hd.hist_rows != hist) return fail(FILARK_EINVAL, "state history length mismatch");
    const size_t need = sizeof(StateHeader) + sizeof(double) * (size_t)C * (size_t)(2 * S) +
                        sizeof(double) * (size_t)C * 3 + sizeof(float) * (size_t)hist * (size_t)C;
    if (bytes < need) return fail(FILARK_EINVAL, "state buffer too small");
    DeviceGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    filark_status st = join_lanes(h, s);
    if (st != FILARK_OK) return st;
    st = zero_state(h, s);
    if (st != FILARK_OK) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "set_state: synchronize");
    const char *p = (const char *)host_buf + sizeof(StateHeader);
    if (S > 0) {
        const int n2 = 2 * S;
        std::vector<double> canon((size_t)C * (size_t)n2);
        std::memcpy(canon.data(), p, sizeof(double) * canon.size());
        p += sizeof(double) * canon.size();
        std::vector<double> m((size_t)C * (size_t)(2 * NS), 0.0);
        for (int c = 0; c < C; ++c)
            for (int r = 0; r < n2; ++r) {
                long double acc = 0;
                for (int q = 0; q < n2; ++q)
                    acc += h->plan.Winv[(size_t)r * n2 + q] * (long double)canon[(size_t)c * n2 + q];
                m[(size_t)c * (2 * NS) + r] = (double)acc;
            }
        if (!h->plan.dense) encode_df_state(m);
        e = cudaMemcpy(h->iir[0], m.data(), sizeof(double) * m.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail_cuda(e, "set_state: copy");
    }
    if (h->det) {
        std::vector<double> d((size_t)C * 4, 0.0);
        for (int c = 0; c < C; ++c) std::memcpy(&d[(size_t)c * 4], p + sizeof(double) * 3 * (size_t)c, sizeof(double) * 3);
        e = cudaMemcpy(h->detst[0], d.data(), sizeof(double) * d.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail_cuda(e, "set_state: copy");
    }
    p += sizeof(double) * 3 * (size_t)C;
    for (int64_t k = 0; k < hist; ++k) {
        const long long nabs = hd.n - hist + k;
        const long long slot = nabs % h->Q;
        e = cudaMemcpy(h->ring + slot * h->ldr, p, sizeof(float) * (size_t)C, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail_cuda(e, "set_state: copy");
        p += sizeof(float) * (size_t)C;
    }
    h->parity = 0;
    h->n = hd.n;
    return FILARK_OK;
}

}  // extern "C"
