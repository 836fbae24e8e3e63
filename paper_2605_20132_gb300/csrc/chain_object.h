// The chain object behind the C-ABI handle, shared by the single-stream API
// (api.cpp) and the batched API (batch.cpp).  Not part of the public API.
#pragma once

#include "filark_internal.h"

struct filark_chain {
    filark_chain_config cfg{};
    std::vector<double> sos;
    filark::Plan plan;
    int device = 0;
    int C = 0, K = 1, hw = 0, HP = 0, Wout = 0, n_tiles = 0;
    bool det = false;
    int ns = 0, nl = 0;
    long long Q = 0, ldr = 0;
    double *iir[2] = {nullptr, nullptr};
    double *detst[2] = {nullptr, nullptr};
    float *ring = nullptr;
    int *status_host = nullptr;   // mapped pinned word written by kernels
    int *status_dev = nullptr;
    int parity = 0;
    long long n = 0;
    filark_status sticky = FILARK_OK;
    float *stage[4] = {nullptr, nullptr, nullptr, nullptr};   // in, ratio, bp, sp
    // pipelined host pushes: per slot staging {in, ratio, bp, sp} and the
    // events that order the input copy, the push and the output copies
    cudaStream_t hcopy_in = nullptr, hcopy_out = nullptr;
    float *astage[FILARK_HOST_SLOTS][4] = {};
    cudaEvent_t ev_in[FILARK_HOST_SLOTS] = {}, ev_comp[FILARK_HOST_SLOTS] = {}, ev_out[FILARK_HOST_SLOTS] = {};
    bool slot_used[FILARK_HOST_SLOTS] = {};
    int aslot = 0;
    float *dense = nullptr;       // dense carry matrices (device)
    filark::ChainParams base{};
    int64_t device_bytes = 0;
    int use_pdl = 1;
    int nbc_fixed = 0;            // blocks per CTA set by the caller, 0 = kNB
    int launch_samples = filark::kMaxLaunchSamples;   // a push is cut into launches of at most this many samples
    // the last filark_chain_tune: candidates and their ms per push
    int n_tuned = 0, tuned_choice = -1;
    int tune_lanes[16] = {}, tune_launch[16] = {}, tune_blocks[16] = {};
    double tune_ms[16] = {};
    // lanes: the channel tiles split into `lanes` contiguous groups, each
    // pushed on an internal stream of its own; a push forks from the caller's
    // stream, and filark_chain_join (or any call that reads or resets the
    // state) joins the lanes back into a caller's stream
    int lanes = 1;
    cudaStream_t lane_s[FILARK_MAX_LANES] = {};
    cudaEvent_t ev_fork = nullptr, ev_lane[FILARK_MAX_LANES] = {};
    bool lanes_pending = false;   // lane work not yet joined into a caller's stream
    // per-tile carried IIR state of all kWT columns, [tiles][kWT][2*NS] per
    // parity, so that a tile never reads a neighbouring tile's (possibly
    // other lane's) state; valid once a lane launch has written it
    double *halo[2] = {nullptr, nullptr};
    bool halo_valid = false;
};

namespace filark {
// zero carried state, ring and counters (enqueued on `stream`)
filark_status chain_zero_state(filark_chain *h, cudaStream_t stream);
// sticky error state / device error word
filark_status chain_check_status(filark_chain *h);
// the argument checks of filark_chain_push_chunk
filark_status chain_validate_push(filark_chain *h, const void *in, int64_t ld_in, int64_t T, const void *ratio,
                                  const void *bp, const void *sp, int64_t ld_out);
}  // namespace filark
