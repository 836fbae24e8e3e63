// Batched chains (include/filark.h, filark_batch_*): many independent streams
// that share one chain configuration, pushed together by ONE persistent
// kernel launch per push.
//
// Each stream is an ordinary chain object (its own carried IIR and detector
// state, history ring, sample counter).  A batched push cuts every stream's
// chunk into units of at most cluster x 256 samples -- the same per-launch
// records filark_chain_push_chunk would enqueue one by one -- and lists one
// work item per (stream, channel tile).  Items are ordered longest chunk first
// and the clusters of a persistent grid take them from a device counter; a
// cluster runs an item's units in order, so each unit reads the state the
// previous one wrote (the tile carries its halo columns' state itself between
// units, since the neighbouring tiles may not have reached that point).  The unit and item tables travel in one pinned staging buffer (two,
// alternating) whose upload and the kernel launch are captured once in a CUDA
// graph per staging buffer; a push fills the tables and replays the graph.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "chain_object.h"
#include "host_trace.h"

using namespace filark;

namespace {

constexpr size_t kAlign = 256;
constexpr int kClusterChoices[] = {1, 2, 4, 8};
constexpr int kDefaultCluster = 8;   // the single-stream kernel's time split
constexpr int kMinBlocksPerCta = 4;  // smallest scan segment per CTA (x 32 samples)
constexpr int kMaxTuned = 16;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }




}  // namespace

struct filark_batch {
    int device = 0;
    std::vector<filark_chain *> chains;
    ChainParams base{};          // static kernel parameters shared by the streams
    int NS = 0;
    bool det = false, dense = false;
    int cluster = kDefaultCluster, n_clusters = 0, use_graph = 1;
    int nbc = kNB;               // scan blocks of 32 samples per CTA
    int64_t max_units = 0, max_items = 0, n_tiles = 0;
    size_t off_items = 0, off_units = 0, desc_bytes = 0;
    size_t staged_bytes = 0;                // bytes of the descriptor block the last push filled
    char *d_desc[2] = {nullptr, nullptr};   // [count | items | units] on the device, per staging buffer
    char *h_stage[2] = {nullptr, nullptr};  // the same, pinned host staging
    cudaEvent_t staged[2] = {nullptr, nullptr};     // staging buffer k uploaded
    cudaEvent_t done[2] = {nullptr, nullptr};       // the kernel that read d_desc[k] finished
    int next = 0;
    cudaStream_t cap = nullptr;             // capture stream (graphs are built here)
    cudaStream_t up = nullptr;              // descriptor uploads of the stream path
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaGraphNode_t upload[2] = {nullptr, nullptr};   // each graph's descriptor copy
    filark_status sticky = FILARK_OK;
    int64_t device_bytes = 0;
    int n_tuned = 0;
    int tune_cluster[kMaxTuned] = {}, tune_clusters[kMaxTuned] = {}, tune_nbc[kMaxTuned] = {};
    double stream_ms = 0.0;     // the best geometry without the graph (last tune)
    double tune_ms[kMaxTuned] = {};
    std::vector<int> order;
    std::vector<int> unit0, nunits;
    std::vector<double *> halo;   // per stream: [2][tiles][kWT][2*NS] tile-private IIR state
    std::vector<double *> detx;   // per stream: [C][4] detector state between the units of one push
};

namespace {

void destroy_graphs(filark_batch *b) {
    for (int k = 0; k < 2; ++k) {
        if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
        if (b->graph[k]) cudaGraphDestroy(b->graph[k]);
        b->exec[k] = nullptr;
        b->graph[k] = nullptr;
        b->upload[k] = nullptr;
    }
}

void free_batch(filark_batch *b) {
    if (!b) return;
    destroy_graphs(b);
    for (cudaEvent_t &e : b->staged)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t &e : b->done)
        if (e) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->up) cudaStreamDestroy(b->up);
    for (char *p : b->h_stage)
        if (p) cudaFreeHost(p);
    for (char *p : b->d_desc)
        if (p) cudaFree(p);
    for (double *p : b->halo)
        if (p) cudaFree(p);
    for (double *p : b->detx)
        if (p) cudaFree(p);
    for (filark_chain *h : b->chains) filark_chain_destroy(h);
    delete b;
}

const BatchItem *dev_items(const filark_batch *b, int k) { return (const BatchItem *)(b->d_desc[k] + b->off_items); }
const ChainUnit *dev_units(const filark_batch *b, int k) { return (const ChainUnit *)(b->d_desc[k] + b->off_units); }
int *dev_ctr(const filark_batch *b, int k) { return (int *)b->d_desc[k]; }

// pdl: launched with programmatic stream serialization (the stream path), so
// that its clusters start while the previous push's last items drain
cudaError_t enqueue_launch(filark_batch *b, int k, cudaStream_t s, bool pdl) {
    ChainParams p = b->base;
    p.pdl = pdl ? 1 : 0;
    return (b->cluster == 1 ? launch_chain_batch_solo : launch_chain_batch)(
        p, b->NS, b->det, b->dense, b->cluster, b->n_clusters, dev_items(b, k),
                              dev_ctr(b, k), dev_units(b, k), s);
}

int max_clusters(const filark_batch *b, int cluster) {
    return cluster == 1 ? batch_max_active_clusters_solo(b->NS, b->det, b->dense, cluster)
                        : batch_max_active_clusters(b->NS, b->det, b->dense, cluster);
}

filark_status build_graphs(filark_batch *b) {
    destroy_graphs(b);
    if (!b->use_graph) return FILARK_OK;
    for (int k = 0; k < 2; ++k) {
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail_cuda_with(e, "batch: begin capture");
        cudaError_t e1 = cudaMemcpyAsync(b->d_desc[k], b->h_stage[k], b->desc_bytes, cudaMemcpyHostToDevice, b->cap);
        cudaError_t e2 = e1 == cudaSuccess ? enqueue_launch(b, k, b->cap, false) : e1;
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(b->cap, &g);
        if (e2 != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail_cuda_with(e2 != cudaSuccess ? e2 : e, "batch: capture of upload + launch");
        }
        b->graph[k] = g;
        // the copy node, whose length each push sets to the bytes it filled
        size_t n = 0;
        e = cudaGraphGetNodes(g, nullptr, &n);
        std::vector<cudaGraphNode_t> nodes(n);
        if (e == cudaSuccess && n > 0) e = cudaGraphGetNodes(g, nodes.data(), &n);
        for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
            cudaGraphNodeType t;
            e = cudaGraphNodeGetType(nodes[i], &t);
            if (e == cudaSuccess && t == cudaGraphNodeTypeMemcpy) b->upload[k] = nodes[i];
        }
        if (e == cudaSuccess && !b->upload[k]) return fail_with(FILARK_ECUDA, "batch: no copy node in the graph");
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[k], g, 0);
        if (e != cudaSuccess) {
            b->exec[k] = nullptr;
            return fail_cuda_with(e, "batch: graph instantiate");
        }
    }
    return FILARK_OK;
}

filark_status set_launch(filark_batch *b, int cluster, int n_clusters, int use_graph, int nbc) {
    if (std::find(std::begin(kClusterChoices), std::end(kClusterChoices), cluster) == std::end(kClusterChoices))
        return fail_with(FILARK_EINVAL, "batch: cluster must be 1, 2, 4 or 8");
    if (nbc < kMinBlocksPerCta || nbc > kNB)
        return fail_with(FILARK_EINVAL, "batch: blocks per CTA must be 4 .. 8");
    if (b->dense && nbc != kNB) return fail_with(FILARK_ENOSYS, "batch: the dense carry uses 8 blocks per CTA");
    int n = n_clusters;
    if (n <= 0) n = max_clusters(b, cluster);
    if (n <= 0) return fail_with(FILARK_ENOSYS, "batch: no cluster of this size fits on the device");
    b->cluster = cluster;
    b->n_clusters = n;
    b->use_graph = use_graph ? 1 : 0;
    b->nbc = nbc;
    // the cross-CTA powers Phi^r of the modal carry depend on the segment
    set_cta_powers(b->chains[0]->plan, nbc, b->base);
    return build_graphs(b);
}

// Fill the staging buffer k for one push; returns the item count.
int stage_push(filark_batch *b, int k, const filark_chunk_desc *d) {
    char *base = b->h_stage[k];
    BatchItem *items = (BatchItem *)(base + b->off_items);
    ChainUnit *units = (ChainUnit *)(base + b->off_units);
    const int n = (int)b->chains.size();
    const int span = kL * b->nbc * b->cluster;
    int nu = 0;
    for (int i = 0; i < n; ++i) {
        filark_chain *h = b->chains[(size_t)i];
        const filark_chunk_desc &c = d[i];
        b->unit0[(size_t)i] = nu;
        b->nunits[(size_t)i] = 0;
        const size_t hstride = (size_t)h->n_tiles * kWT * (size_t)(2 * b->NS);
        double *hs = b->halo[(size_t)i];
        // Every unit of this push runs in the same launch, and a tile's first
        // unit reads its halo columns from the neighbouring tiles' per-channel
        // state iir[P0]; so no unit writes iir[P0]: the intermediate units
        // carry the IIR state in the tile-private halo buffers only, the last
        // writes iir[P0 ^ 1].  The detector state (each tile's own channels)
        // steps through det[P0] -> ... -> det[P0 ^ 1], alternating with a
        // spare buffer so that the last unit lands in det[P0 ^ 1].
        const int P0 = h->parity;
        const int n_u = (int)((c.n_samples + span - 1) / span);
        auto det_buf = [&](int j) -> double * {
            if (j == 0) return h->detst[P0];
            return ((n_u - j) % 2 == 0) ? h->detst[P0 ^ 1] : b->detx[(size_t)i];
        };
        for (int64_t done = 0; done < c.n_samples;) {
            const int Tl = (int)std::min<int64_t>(c.n_samples - done, span);
            const int j = b->nunits[(size_t)i];
            ChainUnit &u = units[nu++];
            u = h->base.u;   // ring, ldr, Q, C
            // tile-private state between the units of this push (unit j reads
            // what unit j-1 wrote; the first reads the per-channel state)
            u.tx0 = 0;   // the batched kernel passes each unit's tile itself
            u.halo_in = (hs && j > 0) ? hs + (size_t)((j - 1) & 1) * hstride : nullptr;
            u.halo_out = (hs && done + Tl < c.n_samples) ? hs + (size_t)(j & 1) * hstride : nullptr;
            u.x = c.d_in + done * c.ld_in;
            u.ldx = c.ld_in;
            u.ratio = c.d_ratio ? c.d_ratio + done * c.ld_out : nullptr;
            u.bp = c.d_bandpass ? c.d_bandpass + done * c.ld_out : nullptr;
            u.sp = c.d_spatial ? c.d_spatial + done * c.ld_out : nullptr;
            u.ldo = c.ld_out;
            u.iir_in = h->iir[P0];
            u.iir_out = j == n_u - 1 ? h->iir[P0 ^ 1] : nullptr;
            u.det_in = det_buf(j);
            u.det_out = det_buf(j + 1);
            u.n0 = h->n;
            set_unit_geometry(h->plan, Tl, b->nbc, u);
            u.slot_n0 = h->Q > 0 ? (int)(h->n % h->Q) : 0;
            u.x_vec4 = (c.ld_in % 4 == 0) && (((uintptr_t)u.x & 15u) == 0);
            bool ov = (c.ld_out % 4 == 0);
            for (float *o : {u.ratio, u.bp, u.sp})
                if (o && ((uintptr_t)o & 15u)) ov = false;
            u.o_vec4 = ov;
            h->n += Tl;
            done += Tl;
            b->nunits[(size_t)i]++;
        }
        if (n_u > 0) h->parity = P0 ^ 1;
    }
    // longest chunk first, then stream order
    std::vector<int> &ord = b->order;
    ord.resize((size_t)n);
    for (int i = 0; i < n; ++i) ord[(size_t)i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return d[a].n_samples > d[c].n_samples; });
    // a push of one unit that needs R < cluster time ranges shares the
    // cluster among cluster / reff tiles, reff = R rounded up to a power of two
    int ni = 0;
    for (int i : ord) {
        const int nu_i = b->nunits[(size_t)i];
        if (nu_i == 0) continue;
        const filark_chain *h = b->chains[(size_t)i];
        int reff = b->cluster;
        if (nu_i == 1) {
            const int R = units[b->unit0[(size_t)i]].R;
            reff = 1;
            while (reff < R) reff <<= 1;
        }
        const int g = b->cluster / reff;
        for (int t = 0; t < h->n_tiles; t += g)
            items[ni++] = BatchItem{b->unit0[(size_t)i], nu_i, t, std::min(g, h->n_tiles - t), reff, {0, 0, 0}};
    }
    ((int *)base)[0] = ni;
    ((int *)base)[1] = 0;   // the kernel's work counter
    b->staged_bytes = b->off_units + sizeof(ChainUnit) * (size_t)nu;
    return ni;
}

filark_status push(filark_batch *b, const filark_chunk_desc *descs, cudaStream_t stream) {
    if (b->sticky != FILARK_OK) return fail_with(FILARK_ESTATE, "batch is in an error state; reset it");
    const int n = (int)b->chains.size();
    for (int i = 0; i < n; ++i) {
        filark_chain *h = b->chains[(size_t)i];
        filark_status st = chain_check_status(h);
        if (st != FILARK_OK) return st;
        const filark_chunk_desc &c = descs[i];
        st = chain_validate_push(h, c.d_in, c.ld_in, c.n_samples, c.d_ratio, c.d_bandpass, c.d_spatial, c.ld_out);
        if (st != FILARK_OK) return fail_with(st, "stream " + std::to_string(i) + ": " + filark_last_error_string());
    }
    const int k = b->next;
    cudaError_t e = cudaEventSynchronize(b->staged[k]);   // the push before last has uploaded this buffer
    if (e != cudaSuccess) return fail_cuda_with(e, "batch: staging event");
    const int ni = stage_push(b, k, descs);
    if (ni == 0) return FILARK_OK;
    // upload only the part of the descriptor block this push filled
    if (b->use_graph) {
        e = cudaGraphExecMemcpyNodeSetParams1D(b->exec[k], b->upload[k], b->d_desc[k], b->h_stage[k],
                                               b->staged_bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaGraphLaunch(b->exec[k], stream);
        if (e == cudaSuccess) e = cudaEventRecord(b->staged[k], stream);
    } else {
        // the upload runs on the side stream once the kernel that last read
        // d_desc[k] (the push before last) is done, so it overlaps the
        // previous push; the launch waits for it and overlaps the previous
        // kernel's tail through programmatic dependent launch
        e = cudaStreamWaitEvent(b->up, b->done[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_desc[k], b->h_stage[k], b->staged_bytes, cudaMemcpyHostToDevice, b->up);
        if (e == cudaSuccess) e = cudaEventRecord(b->staged[k], b->up);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, b->staged[k], 0);
        if (e == cudaSuccess) e = enqueue_launch(b, k, stream, true);
        if (e == cudaSuccess) e = cudaEventRecord(b->done[k], stream);
    }
    if (e != cudaSuccess) {
        b->sticky = FILARK_ECUDA;
        for (filark_chain *h : b->chains) h->sticky = FILARK_ECUDA;
        return fail_cuda_with(e, "batch: launch");
    }
    b->next ^= 1;
    return FILARK_OK;
}

// Wait until no upload reads a staging buffer and no kernel reads a device
// descriptor block (before the launch settings change).
cudaError_t wait_idle(filark_batch *b) {
    for (cudaEvent_t ev : b->staged) {
        const cudaError_t e = cudaEventSynchronize(ev);
        if (e != cudaSuccess) return e;
    }
    for (cudaEvent_t ev : b->done) {
        const cudaError_t e = cudaEventSynchronize(ev);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

filark_status reset(filark_batch *b, cudaStream_t stream) {
    for (filark_chain *h : b->chains) {
        filark_status st = chain_zero_state(h, stream);
        if (st != FILARK_OK) return st;
    }
    b->sticky = FILARK_OK;
    return FILARK_OK;
}

}  // namespace

extern "C" {

filark_status filark_batch_create(const filark_chain_config *cfg, int n_streams, const int32_t *n_channels,
                                  int cuda_device, filark_batch **out) {
    if (!out) return fail_with(FILARK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg || !n_channels) return fail_with(FILARK_EINVAL, "config or n_channels is NULL");
    if (n_streams < 1) return fail_with(FILARK_EINVAL, "n_streams must be >= 1");
    filark_batch *b = new (std::nothrow) filark_batch();
    if (!b) return fail_with(FILARK_ENOMEM, "host allocation failed");
    b->device = cuda_device;
    for (int i = 0; i < n_streams; ++i) {
        filark_chain_config c = *cfg;
        c.n_channels = n_channels[i];
        filark_chain *h = nullptr;
        filark_status st = filark_chain_create(&c, cuda_device, &h);
        if (st != FILARK_OK) {
            const std::string msg = "stream " + std::to_string(i) + ": " + filark_last_error_string();
            free_batch(b);
            return fail_with(st, msg);
        }
        h->use_pdl = 0;
        b->chains.push_back(h);
        b->device_bytes += h->device_bytes;
        double *hs = nullptr;
        if (h->plan.NS > 0) {
            const size_t bytes = sizeof(double) * 2 * (size_t)h->n_tiles * kWT * (size_t)(2 * h->plan.NS);
            DeviceGuard g(cuda_device);
            if (cudaMalloc(&hs, bytes) != cudaSuccess) {
                cudaGetLastError();
                free_batch(b);
                return fail_with(FILARK_ENOMEM, "batch create: halo state allocation");
            }
            b->device_bytes += (int64_t)bytes;
        }
        b->halo.push_back(hs);
        double *dx = nullptr;
        if (h->det) {
            DeviceGuard g(cuda_device);
            if (cudaMalloc(&dx, sizeof(double) * 4 * (size_t)h->C) != cudaSuccess) {
                cudaGetLastError();
                free_batch(b);
                return fail_with(FILARK_ENOMEM, "batch create: detector state allocation");
            }
            b->device_bytes += (int64_t)(sizeof(double) * 4 * (size_t)h->C);
        }
        b->detx.push_back(dx);
        // units are at least kMinBlocksPerCta x 32 samples
        b->max_units += (std::min<int64_t>(cfg->max_chunk, INT32_MAX) + kL * kMinBlocksPerCta - 1) /
                        (kL * kMinBlocksPerCta);
        b->max_items += h->n_tiles;
    }
    b->n_tiles = b->max_items;
    const filark_chain *h0 = b->chains[0];
    b->base = h0->base;
    std::memset(&b->base.u, 0, sizeof(b->base.u));
    b->base.pdl = 0;
    b->NS = h0->plan.NS;
    b->det = h0->det;
    b->dense = h0->plan.dense;
    b->unit0.assign((size_t)n_streams, 0);
    b->nunits.assign((size_t)n_streams, 0);
    b->off_items = kAlign;
    b->off_units = align_up(b->off_items + sizeof(BatchItem) * (size_t)b->max_items);
    b->desc_bytes = b->off_units + sizeof(ChainUnit) * (size_t)b->max_units;

    DeviceGuard dg(cuda_device);
    if (!dg.ok) {
        free_batch(b);
        return fail_with(FILARK_ECUDA, "cudaSetDevice failed for device " + std::to_string(cuda_device));
    }
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc(&b->d_desc[k], b->desc_bytes);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaHostAlloc(&b->h_stage[k], b->desc_bytes, cudaHostAllocDefault);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&b->staged[k], cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&b->done[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->up, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_batch(b);
        return fail_cuda_with(e, "batch create: allocation");
    }
    b->device_bytes += 2 * (int64_t)b->desc_bytes;
    for (int k = 0; k < 2; ++k) std::memset(b->h_stage[k], 0, b->desc_bytes);
    filark_status st = set_launch(b, kDefaultCluster, 0, 1, kNB);
    if (st != FILARK_OK) {
        const std::string msg = filark_last_error_string();
        free_batch(b);
        return fail_with(st, msg);
    }
    *out = b;
    return FILARK_OK;
}

filark_status filark_batch_push(filark_batch *b, const filark_chunk_desc *descs, filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_batch_push");
    if (!b) return fail_with(FILARK_EINVAL, "batch is NULL");
    if (!descs) return fail_with(FILARK_EINVAL, "descs is NULL");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    return push(b, descs, (cudaStream_t)stream);
}

filark_status filark_batch_set_launch(filark_batch *b, int cluster, int n_clusters, int use_graph) {
    if (!b) return fail_with(FILARK_EINVAL, "batch is NULL");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    // the staging buffers may still be read by an earlier upload
    const cudaError_t e = wait_idle(b);
    if (e != cudaSuccess) return fail_cuda_with(e, "batch: staging event");
    return set_launch(b, cluster, n_clusters, use_graph, b->nbc);
}

filark_status filark_batch_set_blocks_per_cta(filark_batch *b, int blocks) {
    if (!b) return fail_with(FILARK_EINVAL, "batch is NULL");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    const cudaError_t e = wait_idle(b);
    if (e != cudaSuccess) return fail_cuda_with(e, "batch: staging event");
    return set_launch(b, b->cluster, b->n_clusters, b->use_graph, blocks);
}

filark_status filark_batch_tune(filark_batch *b, const filark_chunk_desc *descs, int timed_pushes,
                                filark_stream_t stream) {
    if (!b || !descs) return fail_with(FILARK_EINVAL, "batch or descs is NULL");
    if (timed_pushes < 1) return fail_with(FILARK_EINVAL, "timed_pushes must be >= 1");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e != cudaSuccess) {
        if (t0) cudaEventDestroy(t0);
        return fail_cuda_with(e, "tune: events");
    }
    filark_status st = FILARK_OK;
    double best = 1e300;
    int best_cluster = b->cluster, best_n = b->n_clusters, best_nbc = b->nbc;
    b->n_tuned = 0;
    // reset, 2 warm-up pushes, then the mean ms of timed_pushes pushes
    auto time_pushes = [&](double &per) -> filark_status {
        filark_status r = reset(b, s);
        for (int w = 0; w < 2 && r == FILARK_OK; ++w) r = push(b, descs, s);
        if (r == FILARK_OK && (e = cudaEventRecord(t0, s)) != cudaSuccess) r = fail_cuda_with(e, "tune: record start");
        for (int q = 0; q < timed_pushes && r == FILARK_OK; ++q) r = push(b, descs, s);
        if (r == FILARK_OK && (e = cudaEventRecord(t1, s)) != cudaSuccess) r = fail_cuda_with(e, "tune: record end");
        if (r == FILARK_OK && (e = cudaEventSynchronize(t1)) != cudaSuccess) r = fail_cuda_with(e, "tune: sync");
        float ms = 0.f;
        if (r == FILARK_OK && (e = cudaEventElapsedTime(&ms, t0, t1)) != cudaSuccess)
            r = fail_cuda_with(e, "tune: elapsed");
        per = (double)ms / timed_pushes;
        return r;
    };
    // scan segments of 8 and 4 blocks per CTA (the dense carry: 8 only) x
    // cluster sizes x one or two grids' worth of resident clusters
    for (int nbc : {kNB, kMinBlocksPerCta}) {
        if (b->dense && nbc != kNB) continue;
        for (int cl : kClusterChoices) {
            const int occ = max_clusters(b, cl);
            if (occ <= 0) continue;
            for (int mult : {1, 2}) {
                if (b->n_tuned >= kMaxTuned) break;
                wait_idle(b);
                st = set_launch(b, cl, occ * mult, 1, nbc);
                double per = 0.0;
                if (st == FILARK_OK) st = time_pushes(per);
                if (st != FILARK_OK) break;
                b->tune_cluster[b->n_tuned] = cl;
                b->tune_clusters[b->n_tuned] = occ * mult;
                b->tune_nbc[b->n_tuned] = nbc;
                b->tune_ms[b->n_tuned] = per;
                b->n_tuned++;
                if (per < best) {
                    best = per;
                    best_cluster = cl;
                    best_n = occ * mult;
                    best_nbc = nbc;
                }
            }
            if (st != FILARK_OK) break;
        }
        if (st != FILARK_OK) break;
    }
    // the fastest geometry once more without the graph: uploads on a side
    // stream and programmatic launches that overlap consecutive pushes
    int best_graph = 1;
    if (st == FILARK_OK) {
        wait_idle(b);
        st = set_launch(b, best_cluster, best_n, 0, best_nbc);
        double per_stream = 0.0;
        if (st == FILARK_OK) st = time_pushes(per_stream);
        if (st == FILARK_OK) {
            b->stream_ms = per_stream;
            if (per_stream < best) best_graph = 0;
        }
    }
    // the timing events are used by time_pushes up to here
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st != FILARK_OK) return st;
    wait_idle(b);
    if (st == FILARK_OK) st = set_launch(b, best_cluster, best_n, best_graph, best_nbc);
    if (st == FILARK_OK) st = reset(b, s);
    if (st == FILARK_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = fail_cuda_with(e, "tune: sync");
    return st;
}

filark_status filark_batch_reset_state(filark_batch *b, filark_stream_t stream) {
    if (!b) return fail_with(FILARK_EINVAL, "batch is NULL");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    return reset(b, (cudaStream_t)stream);
}

filark_status filark_batch_sync_status(filark_batch *b, filark_stream_t stream) {
    if (!b) return fail_with(FILARK_EINVAL, "batch is NULL");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        b->sticky = FILARK_ECUDA;
        return fail_cuda_with(e, "batch: synchronize");
    }
    if (b->sticky != FILARK_OK) return fail_with(FILARK_ESTATE, "batch is in an error state; reset it");
    for (filark_chain *h : b->chains) {
        filark_status st = chain_check_status(h);
        if (st != FILARK_OK) return st;
    }
    return FILARK_OK;
}

filark_status filark_batch_get_info(const filark_batch *b, filark_batch_info *out) {
    if (!b || !out) return fail_with(FILARK_EINVAL, "batch or out is NULL");
    std::memset(out, 0, sizeof(*out));
    out->n_streams = (int32_t)b->chains.size();
    out->cluster = b->cluster;
    out->n_clusters = b->n_clusters;
    out->use_graph = b->use_graph;
    out->n_tiles = b->n_tiles;
    out->device_bytes = b->device_bytes;
    out->n_tuned = b->n_tuned;
    for (int i = 0; i < b->n_tuned; ++i) {
        out->tune_cluster[i] = b->tune_cluster[i];
        out->tune_clusters[i] = b->tune_clusters[i];
        out->tune_ms[i] = b->tune_ms[i];
        out->tune_blocks[i] = b->tune_nbc[i];
    }
    out->blocks_per_cta = b->nbc;
    out->tune_stream_ms = b->stream_ms;
    return FILARK_OK;
}

filark_status filark_batch_stream(filark_batch *b, int i, filark_chain **out) {
    if (!b || !out) return fail_with(FILARK_EINVAL, "batch or out is NULL");
    if (i < 0 || i >= (int)b->chains.size()) return fail_with(FILARK_EINVAL, "stream index out of range");
    *out = b->chains[(size_t)i];
    return FILARK_OK;
}

filark_status filark_batch_destroy(filark_batch *b) {
    if (!b) return FILARK_OK;
    DeviceGuard dg(b->device);
    wait_idle(b);
    free_batch(b);
    return FILARK_OK;
}

}  // extern "C"
