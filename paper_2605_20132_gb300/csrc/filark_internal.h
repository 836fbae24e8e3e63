// Internal declarations shared by the host planner, the C-ABI layer and the
// CUDA kernels of the chunked DAS filter chain.  Not part of the public API.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/filark.h"

namespace filark {

// ---------------------------------------------------------------------------
// Kernel geometry.
//
// One thread block (CTA) owns a tile of kWT channels (output channels plus a
// halo on both sides) and kNB time blocks of kL samples.  The IIR stage runs
// one thread per (channel, time block); the CTAs of one tile that cover
// consecutive time ranges of a launch form one thread-block cluster (at most
// kMaxCluster CTAs), and pass their IIR carries and detector sums through
// distributed shared memory.
// ---------------------------------------------------------------------------
constexpr int kL = 32;                    // samples per time block
constexpr int kNB = 8;                    // time blocks per CTA (at most; a launch may use fewer)
constexpr int kWT = 64;                   // channels per CTA tile (incl. halo)
constexpr int kThreads = kWT * kNB;       // 512 threads: one per (channel, block)
constexpr int kTileRows = kL * kNB;       // 256 samples per CTA
constexpr int kMaxCluster = 8;            // CTAs per cluster (time split, portable size)
constexpr int kCTAsPerSM = 2;             // occupancy target (registers <= 64/thread)
constexpr int kMaxLaunchSamples = kTileRows * kMaxCluster;  // 2048 samples per launch
constexpr int kMaxSlots = 8;              // 2x2 state slots per channel (= sections)
constexpr int kDenseDim = 2 * kMaxSlots;  // 16: dense state dimension
constexpr int kDenseMats = kL + kMaxCluster;  // A^1..A^L, Phi^0..Phi^(kMaxCluster-1)

// FP32 tables of one chain.  They travel in the kernel parameter block, which
// lives in the constant bank, so the fully unrolled contractions read them as
// FFMA constant operands (no load instructions).
struct Tables32 {
    float h[kL];                        // impulse response h[0..L)
    float K[kL][2 * kMaxSlots];         // K[i][r]: input i of a block -> end state r
    float G[kL][2 * kMaxSlots];         // G[k][r]: start state r -> output k
    float M[kMaxSlots][4];              // per slot, M^L as {m00, m01, m10, m11}
};

// What changes from one launch to the next (and, in a batch, from one stream
// to another): buffers, carried-state parity, position in the stream and the
// launch geometry with its ragged-end transitions.
struct ChainUnit {
    const float *x;                     // launch input, row 0 = first sample
    long long ldx;
    float *ratio, *bp, *sp;             // launch outputs (row 0 = first sample)
    long long ldo;
    // [C][2*NS] carried IIR state in the internal basis, 8 bytes per entry:
    // modal carries store double-float {hi, lo} float pairs, the dense carry
    // stores FP64
    const double *iir_in;
    double *iir_out;                    // NULL: the owned channels' state is not written (a batched
                                        // push's units before its last)
    const double *det_in;               // [C][4] {sta_sum, lta_sum, 1 + index of last nonzero cf (0 = none), 0}
    double *det_out;
    // Batched pushes run a stream's units back to back in one cluster, so a
    // tile cannot wait for its neighbours' end states: it carries the state of
    // all kWT columns (halo included) itself, [tiles][kWT][2*NS], between the
    // units of one push.  NULL: read iir_in / write only the owned channels.
    const double *halo_in;
    double *halo_out;
    float *ring;                        // [Q][ldr] cf history
    long long ldr;
    long long n0;                       // global index of the launch's first sample
    int Q;                              // ring length in samples
    int slot_n0;                        // n0 mod Q
    int C, T, nblk, Lr, R;
    int nbc;                            // blocks per CTA (<= kNB): CTA r covers blocks [r nbc, r nbc + nbc)
    int tx0;                            // channel tile of grid.x = 0 (a launch may cover a tile range)
    int x_vec4, o_vec4;                 // float4 access allowed (input, outputs)
    // trigger summaries fused into the detector (chain_fwd_kernel<..., TRIG>):
    // [blocks of the launch][C] packed segment summaries, row 0 = the launch's
    // first 32-sample block
    unsigned *trig_summ;
    // transition over the launch's last CTA, and PhiTot = PhiLast * Phi^(R-1)
    // (launch start -> launch end), as double-float hi/lo pairs
    float PhiLastHi[kMaxSlots][4], PhiLastLo[kMaxSlots][4];
    float PhiTotHi[kMaxSlots][4], PhiTotLo[kMaxSlots][4];
    float Mr32[kMaxSlots][4];           // M^Lr of the ragged last block (Lr < L), FP32
};

// Everything else is fixed for a chain (for a batch: shared by its streams).
struct ChainParams {
    Tables32 tab;
    float PhiPow32[kMaxCluster][kMaxSlots][4]; // Phi^r = M^(L*nbc*r), FP32, for the launch's nbc
    int hw, HP, Wout;
    int ns, nl;
    float ratio_scale;                  // nl / ns
    float trig_on, trig_off;            // trigger thresholds (floats >= the doubles) for TRIG launches
    int all32;                          // keep carries in FP32 everywhere (comparison)
    int pdl;                            // launched with programmatic stream serialization
    // dense carry (FILARK_PREC_DENSE64, or ALL32 without a modal basis):
    // matrices 0..31 = A^1..A^32, 32..39 = Phi^0..Phi^7, each as double-float
    // entries in the lane layout [kDenseDim][8] float4 (plan.cpp,
    // dense_lane_layout)
    const float *dense;
    ChainUnit u;                        // the launch (single-stream kernel)
};

// One work item of the batched kernel: n_tiles channel tiles of one stream,
// whose push is the units [unit0, unit0 + n_units) run in order by one
// cluster; cluster ranks [k reff, (k + 1) reff) run tile `tile + k`.
struct BatchItem {
    int unit0, n_units;
    int tile, n_tiles;   // tiles tile .. tile + n_tiles - 1 of the stream
    int reff;            // cluster ranks per tile (a power of two dividing the cluster)
    int pad[3];
};

// ---------------------------------------------------------------------------
// Host planner.
// ---------------------------------------------------------------------------
struct Plan {
    int S = 0;                // sections
    int NS = 0;               // slots the kernel runs (S padded to 2, 4 or 8; 0 = no IIR)
    int mode = FILARK_PREC_MODAL32;
    bool dense = false;       // dense double-float carry in the canonical basis
    // dense matrices (see ChainParams::dense), host copy
    std::vector<float> dense_mats;
    double kappa = 0.0;       // condition number estimate of the modal basis
    double probe_err = 0.0;   // FP32 emulation error on the probe signal
    Tables32 tab{};
    // Per slot: kind (0 = complex pair a +- ib, 1 = two real poles p, q).
    int slot_kind[kMaxSlots] = {};
    long double slot_a[kMaxSlots] = {}, slot_b[kMaxSlots] = {};
    // Real modal basis: canonical state s = W m, m = Winv s (2S x 2S, row-major).
    std::vector<long double> W, Winv;
    // M^n per slot in FP64 (row-major 2x2), for any n >= 0.
    void slot_power(int n, double out[kMaxSlots][4]) const;
    // Memoised slot_power for 0 <= n <= kTileRows (the per-launch transitions).
    const double (*power_cached(int n) const)[4];
    mutable std::vector<double> pow_cache;     // (kTileRows + 1) x kMaxSlots x 4
    mutable std::vector<char> pow_have;
    // Phi^r = M^(L*nbc*r) for 0 <= r < kMaxCluster, 1 <= nbc <= kNB.
    const double (*power_cached_cta(int nbc, int r) const)[4];
    mutable std::vector<double> cta_cache;     // (kNB + 1) x kMaxCluster x kMaxSlots x 4
    mutable std::vector<char> cta_have;
};

// Message returned by filark_last_error_string on this thread.
void set_last_error(const std::string &msg);

// Records msg as this thread's last error and returns st.
inline filark_status fail_with(filark_status st, const std::string &msg) {
    set_last_error(msg);
    return st;
}

// Clears the CUDA error state, records "what: <CUDA message>" and returns
// FILARK_ECUDA.
inline filark_status fail_cuda_with(cudaError_t e, const char *what) {
    cudaGetLastError();
    set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    return FILARK_ECUDA;
}

// Makes `dev` the current device and restores the caller's on scope exit.
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
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};

// Validate and normalise the SOS (a0 != 0, finite, stable), and build the
// plan.  Returns FILARK_OK or an error with a message in *err.
filark_status make_plan(const double *sos, int S, int precision, Plan *plan, std::string *err);

// Butterworth bandpass design (host, long double internally).
filark_status design_butter_bandpass(int order, double f1, double f2, double fs, double *sos,
                                     std::string *err);

// Fill the launch geometry of a unit of Tl samples with nbc blocks per CTA
// (1 <= Tl <= kL * nbc * kMaxCluster) and its ragged-end transitions.
void set_unit_geometry(const Plan &plan, int Tl, int nbc, ChainUnit &u);


// p.PhiPow32 for nbc blocks per CTA.
void set_cta_powers(const Plan &plan, int nbc, ChainParams &p);

// Static kernel parameters of a chain (tables, transitions, geometry).
void set_static_params(const Plan &plan, int hw, int HP, int Wout, int ns, int nl, const float *dense_dev,
                       ChainParams &p);

// ---------------------------------------------------------------------------
// Kernel launch (chain_kernel.cu).  Enqueues one launch of <= kMaxLaunchSamples.
// ---------------------------------------------------------------------------
cudaError_t launch_chain(const ChainParams &p, int NS, bool detector, bool dense, int n_tiles,
                         cudaStream_t stream);

size_t chain_smem_bytes(bool dense);
// The same launch with the detector writing the trigger summaries too
// (p.u.trig_summ, p.trig_on / trig_off); detector chains only.
cudaError_t launch_chain_trig(const ChainParams &p, int NS, bool dense, int n_tiles, cudaStream_t stream);
cudaError_t configure_chain_trig_kernels();   // chain_kernel_trig.cu

// A trigger as the chain's detector sees it when it writes the trigger
// summaries itself (trigger.cu): the summary buffer the next push fills
// ([ceil(max_chunk / 32)][C]), the thresholds as floats, the sizes.
struct TriggerFusion {
    unsigned *summ;
    float on, off;
    int C;
    long long max_chunk;
    int overlap;        // the trigger's scan and emission run on its own stream
};
// Makes `stream` wait until the summary buffer of the next push is free and
// describes it.
filark_status trigger_fusion_begin(filark_trigger *t, cudaStream_t stream, TriggerFusion &out);
// The rest of filark_trigger_push after the summaries: scan and emission.
// In the overlap mode the scan also waits for deps[0 .. n_deps) (the lanes of
// a chain push whose detector wrote the summaries).
filark_status trigger_push_summarized(filark_trigger *t, const float *d_ratio, long long ld, long long n_samples,
                                      filark_trigger_record *d_records, long long capacity,
                                      unsigned long long *d_count, cudaStream_t stream,
                                      const cudaEvent_t *deps = nullptr, int n_deps = 0);


// The batched kernel: a persistent grid of `n_clusters` clusters of `cluster`
// CTAs (time ranges) takes the items in order from a device counter.
// d_ctr[0] = item count, d_ctr[1] = next item (0 at launch); both live in
// device memory so that a captured graph can be replayed with other tables.
// The _solo forms run clusters of one CTA with block barriers in the body
// (chain_batch_solo.cu); batch.cpp uses them whenever cluster == 1.
cudaError_t launch_chain_batch(const ChainParams &p, int NS, bool detector, bool dense, int cluster,
                               int n_clusters, const BatchItem *d_items, int *d_ctr,
                               const ChainUnit *d_units, cudaStream_t stream);
cudaError_t launch_chain_batch_solo(const ChainParams &p, int NS, bool detector, bool dense, int cluster,
                                    int n_clusters, const BatchItem *d_items, int *d_ctr,
                                    const ChainUnit *d_units, cudaStream_t stream);

// Function attributes of the batched kernels (called by configure_chain_kernels).
cudaError_t configure_batch_kernels();
cudaError_t configure_batch_kernels_solo();

// Clusters of `cluster` CTAs that can be resident at once (0 if unknown).
int batch_max_active_clusters(int NS, bool detector, bool dense, int cluster);
int batch_max_active_clusters_solo(int NS, bool detector, bool dense, int cluster);

// Set the kernels' function attributes on the current device (call once per
// device before the first launch).
cudaError_t configure_chain_kernels();

}  // namespace filark
