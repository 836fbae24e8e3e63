// Device code of the fused chain, shared by the single-stream kernel
// (chain_kernel.cu) and the batched persistent kernel (chain_batch.cu).
//
// Fused chunked DAS chain kernel for sm_103a: causal SOS bandpass (block
// state-space form, see plan.cpp), spatial running mean, STA/LTA detector.
//
// Work decomposition of one launch (<= 2048 samples of every channel):
//   grid.x  = channel tiles; a tile is kWT = 64 consecutive channels of which
//             Wout are outputs and HP on each side are halo (the spatial mean
//             of an output channel needs its neighbours' bandpass output, so
//             the halo channels' IIR is computed again by the neighbour tile --
//             the overlap-aware halo expansion of Sec. 3.4);
//   grid.y  = R time ranges of nbc <= kNB blocks x kL samples; the R CTAs of a tile
//             form one thread-block cluster and exchange their IIR carries and
//             detector sums through distributed shared memory.
//
// Per CTA (512 threads):
//   0. load the input tile [256 samples][64 channels] into shared memory;
//   1. per (channel, block): local FIR response y_loc = T_L x and the block's
//      end state e = K x from zero state (FP32, tables are FFMA constant
//      operands);
//   2. per (channel, slot): carry scan m_{j+1} = M m_j + e_j -- FP32 inside the
//      CTA and from the CTAs of the cluster, double-float for the state carried
//      across launches (the dense mode carries in FP64);
//   3. fix-up y_bp = y_loc + G m_j, written back in place;
//   4. spatial mean over the 2h+1 neighbouring columns, cf = y_sp^2, written to
//      the detector's history ring and kept in place;
//   5. STA/LTA: exact (compensated) block sums, double-float scan across
//      blocks and CTAs, then FP32 running sums inside each block and the ratio.
//
// Consecutive launches on a stream overlap through programmatic dependent
// launch: phases 0-1 only read the caller's input, so a launch starts them
// while the previous one drains, and waits for it before touching the state.
#pragma once

#include <climits>
#include <type_traits>

#include <cooperative_groups.h>

#include "filark_internal.h"

namespace cg = cooperative_groups;

namespace filark {

namespace {

__device__ __forceinline__ void cluster_sync_release_acquire() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// The two halves of a cluster barrier, for work in between: arrive (release:
// this CTA's earlier writes become visible to the cluster; relaxed: no
// ordering) and wait (acquire).  Every thread of the CTA executes each.
__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// The body's barriers.  A tile whose time ranges are a whole cluster of one
// CTA (SOLO: the batched kernel with clusters of 1) exchanges nothing through
// distributed shared memory, so a block barrier does: the split arrive is
// dropped and the wait becomes the barrier.  (The batched kernel fences
// global memory once per unit instead; see chain_batch.cu.)
template <bool SOLO>
__device__ __forceinline__ void body_sync() {
    if constexpr (SOLO) __syncthreads();
    else cluster_sync_release_acquire();
}
template <bool SOLO>
__device__ __forceinline__ void body_arrive_release() {
    if constexpr (!SOLO) cluster_arrive_release();
}
template <bool SOLO>
__device__ __forceinline__ void body_arrive_relaxed() {
    if constexpr (!SOLO) cluster_arrive_relaxed();
}
template <bool SOLO>
__device__ __forceinline__ void body_wait() {
    if constexpr (SOLO) __syncthreads();
    else cluster_wait_acquire();
}

// 1 / x to about one ulp (the hardware approximation, subnormals flushed)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

__device__ __forceinline__ void pdl_wait() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

// s + v for s, v >= 0 with the rounding error kept in c (Fast2Sum on the larger
// operand), so a block sum of non-negative values is carried as s + c with an
// error of order eps^2 instead of eps.
__device__ __forceinline__ void acc_nonneg(float &s, float &c, float v) {
    const float t = s + v;
    const float big = fmaxf(s, v), small = fminf(s, v);
    c += small - (t - big);
    s = t;
}

// Double-float (hi + lo) arithmetic for the carried IIR state and the
// detector's carried sums: error-free additions (Knuth's TwoSum) and FMA-based
// products keep ~48 significant bits without the FP64 pipe (1/64 rate).
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float err = (a.hi - (s - bb)) + (b.hi - bb);
    const float lo = err + (a.lo + b.lo);
    const float hi = s + lo;
    return DF{hi, lo - (hi - s)};
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
// a * b with the leading product exact (FMA), ~2^-46 relative
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float hi = p + e;
    return DF{hi, e - (hi - p)};
}
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    const float hi = p + e;
    return DF{hi, e - (hi - p)};
}
// a + c for a, c >= 0 held as compensated sums (s, comp): exact as DF
__device__ __forceinline__ DF df_from_sum(float s, float comp) {
    const float hi = s + comp;
    return DF{hi, comp - (hi - s)};
}

// shared memory carve-up (floats)
constexpr int kTileFloats = kTileRows * kWT;                 // 16384
constexpr int kEFloats = kNB * 2 * kMaxSlots * kWT;          // 8192
constexpr int kERFloats = 2 * kMaxSlots * kWT;               // 1024
constexpr int kAggFloats = 2 * kMaxSlots * kWT;              // 1024 (also holds 3 x 64 doubles)
constexpr int kSmemFloats = kTileFloats + kEFloats + kERFloats + kAggFloats;
// the dense carry needs a double-float aggregate [16][kWT] in place of AGG
// (its running state lives in registers)
constexpr int kAggDenseFloats = kDenseDim * kWT * 2;          // 2048
constexpr int kSmemFloatsDense = kTileFloats + kEFloats + kERFloats + kAggDenseFloats;
static_assert(2 * (kSmemFloatsDense * 4 + 1024) <= 228 * 1024, "two dense CTAs per SM");

// detector overlays on the E region (free after the IIR fix-up); offsets in floats
constexpr int kDetDS = 0;                                    // DF [kNB][kWT]
constexpr int kDetDL = kDetDS + kNB * kWT * 2;               // DF [kNB][kWT]
constexpr int kDetBS = kDetDL + kNB * kWT * 2;               // DF [kNB][kWT]
constexpr int kDetBL = kDetBS + kNB * kWT * 2;               // DF [kNB][kWT]
constexpr int kDetLZ = kDetBL + kNB * kWT * 2;               // int [kNB][kWT] last nonzero row
constexpr int kDetBZ = kDetLZ + kNB * kWT;                   // int [kNB][kWT] its running max
static_assert(kDetBZ + kNB * kWT <= kEFloats, "detector overlays must fit in the E region");

constexpr int kNoNonzero = INT_MIN / 2;   // "no nonzero cf" as a relative row index
constexpr int kRowStep = kThreads / 16;   // rows covered by one pass of the spatial phase
constexpr int kRowIters = kTileRows / kRowStep;


// Stores of one 4-channel group of a row: the spatial tap and, with the
// detector, cf = y_sp^2 into the history ring.
template <bool DET>
__device__ __forceinline__ void store_group(const ChainUnit &cu, int row, int row0, int cch, int slot_r0,
                                            bool full_group, const float (&ysp)[4], float (&cf)[4]) {
    if (cu.sp) {
        float *dst = cu.sp + (long long)(row0 + row) * cu.ldo + cch;
        if (cu.o_vec4 && full_group) {
            *reinterpret_cast<float4 *>(dst) = make_float4(ysp[0], ysp[1], ysp[2], ysp[3]);
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (cch + u < cu.C) dst[u] = ysp[u];
        }
    }
    if (DET) {
#pragma unroll
        for (int u = 0; u < 4; ++u) cf[u] = ysp[u] * ysp[u];
        int slot = slot_r0 + row;
        if (slot >= cu.Q) slot -= cu.Q;
        float *dst = cu.ring + (long long)slot * cu.ldr + cch;
        if (full_group) {
            *reinterpret_cast<float4 *>(dst) = make_float4(cf[0], cf[1], cf[2], cf[3]);
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (cch + u < cu.C) dst[u] = cf[u];
        }
    }
}

// With the detector on, cf replaces y_bp in the tile once every thread has
// read its windows (rows past the end get cf = 0).  Called by all threads.
template <bool DET>
__device__ __forceinline__ void store_cf_in_place(float *tile, int ro, int rows, int q0, bool gact,
                                                  const float (&cfv)[kRowIters][4]) {
    if (!DET) return;
    __syncthreads();
    if (gact) {
#pragma unroll
        for (int it = 0; it < kRowIters; ++it) {
            const int row = ro + kRowStep * it;
            *reinterpret_cast<float4 *>(&tile[row * kWT + q0]) = row < rows
                ? make_float4(cfv[it][0], cfv[it][1], cfv[it][2], cfv[it][3])
                : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// Spatial mean of 4 output columns q0..q0+3 for the rows ro, ro+32, ... of the
// tile, window half-width HW <= 4 known at compile time (halo HP = 4, or 0 when
// HW = 0): the 12 (or 4) columns around the group come in with aligned float4
// loads, which are free of bank conflicts.
template <int HW, bool DET>
__device__ __forceinline__ void spatial_rows(const ChainUnit &cu, float *tile, int ro, int rows, int q0,
                                             int row0, int cch, int slot_r0, bool full_group, bool gact,
                                             const float (&inv)[4]) {
    constexpr int H = HW == 0 ? 0 : 4;              // halo columns loaded on each side
    float cfv[kRowIters][4];
#pragma unroll
    for (int it = 0; it < kRowIters; ++it) {
        const int row = ro + kRowStep * it;
        cfv[it][0] = cfv[it][1] = cfv[it][2] = cfv[it][3] = 0.f;
        if (gact && row < rows) {
            float v[4 + 2 * H];
            const float4 *tr = reinterpret_cast<const float4 *>(tile + row * kWT + q0 - H);
#pragma unroll
            for (int f = 0; f < (4 + 2 * H) / 4; ++f) {
                const float4 t = tr[f];
                v[4 * f + 0] = t.x;
                v[4 * f + 1] = t.y;
                v[4 * f + 2] = t.z;
                v[4 * f + 3] = t.w;
            }
            float sacc = 0.f;
#pragma unroll
            for (int q = H - HW; q <= H + HW; ++q) sacc += v[q];
            float ysp[4];
            ysp[0] = sacc * inv[0];
#pragma unroll
            for (int u = 1; u < 4; ++u) {
                sacc += v[H + u + HW] - v[H + u - 1 - HW];
                ysp[u] = sacc * inv[u];
            }
            store_group<DET>(cu, row, row0, cch, slot_r0, full_group, ysp, cfv[it]);
        }
    }
    store_cf_in_place<DET>(tile, ro, rows, q0, gact, cfv);
}

// Same for any halo width (hw runtime, columns read one by one).
template <bool DET>
__device__ __forceinline__ void spatial_rows_generic(const ChainParams &p, const ChainUnit &cu, float *tile, int ro, int rows,
                                                  int q0, int row0, int cch, int slot_r0, bool full_group,
                                                  bool gact, const float (&inv)[4]) {
    float cfv[kRowIters][4];
#pragma unroll
    for (int it = 0; it < kRowIters; ++it) {
        const int row = ro + kRowStep * it;
        cfv[it][0] = cfv[it][1] = cfv[it][2] = cfv[it][3] = 0.f;
        if (gact && row < rows) {
            const float *tr = tile + row * kWT;
            float sacc = 0.f;
            for (int q = q0 - p.hw; q <= q0 + p.hw; ++q) sacc += tr[q];
            float ysp[4];
            ysp[0] = sacc * inv[0];
            for (int u = 1; u < 4; ++u) {
                sacc += tr[q0 + u + p.hw] - tr[q0 + u - 1 - p.hw];
                ysp[u] = sacc * inv[u];
            }
            store_group<DET>(cu, row, row0, cch, slot_r0, full_group, ysp, cfv[it]);
        }
    }
    store_cf_in_place<DET>(tile, ro, rows, q0, gact, cfv);
}

// Dense carry.  The state of one tile column (n = 2NS rows in the canonical
// basis) is held as double-float pairs by 8 lanes of one warp: lane w < NS
// holds rows w and n-1-w (lanes w >= NS hold zeros).  The transition powers
// are block lower triangular, so row w < NS needs the state rows q < NS and
// row n-1-w all n of them: 3NS products per lane and step, whatever w is.
struct DenseRows {
    DF lo, hi;   // rows w and n-1-w
};

// s + t += m * v for double-float m and v, the sum kept unnormalised: the
// leading products are split exactly (TwoProduct by FMA) and summed exactly
// (TwoSum) into s; their rounding errors and the cross terms go into t, as in
// the compensated dot product of Ogita, Rump and Oishi (2005).  The _rn forms
// keep the compiler from fusing the steps whose rounding is meant.
__device__ __forceinline__ void df_dot_step(float &s, float &t, float mh, float ml, float vh, float vl) {
    const float p = __fmul_rn(mh, vh);
    const float pe = fmaf(mh, vh, -p);
    const float s2 = __fadd_rn(s, p);
    const float bb = __fsub_rn(s2, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bb)), __fsub_rn(p, bb));
    t = fmaf(mh, vl, t);
    t = fmaf(ml, vh, t);
    t = __fadd_rn(t, __fadd_rn(pe, err));
    s = s2;
}
__device__ __forceinline__ DF df_norm(float s, float t) {
    const float hi = __fadd_rn(s, t);
    return DF{hi, __fsub_rn(t, __fsub_rn(hi, s))};
}
__device__ __forceinline__ DF df_from_double(double v) {
    const float hi = __double2float_rn(v);
    return DF{hi, __double2float_rn(v - (double)hi)};
}

// One step of the dense carry for the 8 lanes of a column: state <- Mx state
// + add, Mx one matrix in the lane layout [n][8] float4 (row w: hi, lo; row
// n-1-w: hi, lo).  The state rows travel by warp shuffles; every lane of the
// warp executes it.  With all32 the result is rounded to FP32 (comparison).
template <int NS>
__device__ __forceinline__ void dense_step(const float4 *__restrict__ Mx, DenseRows &st, DF add_lo, DF add_hi,
                                           int w, int lane_base, bool all32) {
    constexpr int n = 2 * NS;
    float sl = add_lo.hi, tl = add_lo.lo, sh = add_hi.hi, th = add_hi.lo;
    // state rows q < NS are the lanes' first rows, q >= NS their second ones
#pragma unroll 4
    for (int q = 0; q < NS; ++q) {
        const float vh = __shfl_sync(0xffffffffu, st.lo.hi, lane_base + q);
        const float vl = __shfl_sync(0xffffffffu, st.lo.lo, lane_base + q);
        const float4 m = __ldg(Mx + q * 8 + w);
        df_dot_step(sh, th, m.z, m.w, vh, vl);
        df_dot_step(sl, tl, m.x, m.y, vh, vl);
    }
    const float2 *Mh = reinterpret_cast<const float2 *>(Mx);
#pragma unroll 4
    for (int q = NS; q < n; ++q) {
        const float vh = __shfl_sync(0xffffffffu, st.hi.hi, lane_base + n - 1 - q);
        const float vl = __shfl_sync(0xffffffffu, st.hi.lo, lane_base + n - 1 - q);
        const float2 m = __ldg(Mh + (q * 8 + w) * 2 + 1);
        df_dot_step(sh, th, m.x, m.y, vh, vl);
    }
    st.lo = df_norm(sl, tl);
    st.hi = df_norm(sh, th);
    if (all32) {
        st.lo.lo = 0.f;
        st.hi.lo = 0.f;
    }
}

// Cluster rank of time range q of this CTA's tile: the tile's time ranges are
// consecutive ranks, this CTA (time range r) among them (the single-stream
// kernel gives a tile the whole cluster; the batched kernel may put several
// tiles of a short push in one cluster).
__device__ __forceinline__ unsigned tile_rank(const cg::cluster_group &cluster, int r, int q) {
    return cluster.block_rank() - (unsigned)r + (unsigned)q;
}

// The work of one CTA: time range r of channel tile `tx` for the launch `cu`.
// Every CTA of the cluster calls it with the same unit; it executes
// chain_cluster_barriers<NS, DET>() cluster barriers.
// Trigger summary of one channel's 32-sample segment (TRIG): the hysteresis
// state s(n) = 1 if R(n) >= on, 0 if R(n) < off, else s(n-1), run from both
// possible entry states on the ratio as it is written; packed as the trigger
// pipeline's scan reads it (bits 0/1 final state from 0/1, bits 2/3 a run
// ends inside when entering with 0/1, bits 4-9 / 10-15 last rise + 1).
struct TrigAuto {
    // kept directly in the packed form (one register): entry 1's state starts at 1
    unsigned w = 2u;
    __device__ __forceinline__ void step(float r, float on, float off, int k) {
        const unsigned set = r >= on, keep = !(r < off);
        const unsigned s0 = w & 1u, s1 = (w >> 1) & 1u;
        const unsigned n0 = set | (keep & s0), n1 = set | (keep & s1);
        const unsigned rise0 = n0 & (s0 ^ 1u), rise1 = n1 & (s1 ^ 1u);
        const unsigned end0 = s0 & (n0 ^ 1u), end1 = s1 & (n1 ^ 1u);
        const unsigned k1 = (unsigned)(k + 1);
        w = (w & ~3u) | n0 | (n1 << 1) | (end0 << 2) | (end1 << 3);
        if (rise0) w = (w & ~(63u << 4)) | (k1 << 4);
        if (rise1) w = (w & ~(63u << 10)) | (k1 << 10);
    }
    __device__ __forceinline__ unsigned packed() const { return w; }
};

template <int NS, bool DET, bool DENSE, bool SOLO = false, bool TRIG = false>
__device__ __forceinline__ void chain_body(const ChainParams &p, const ChainUnit &cu, const int tx, const int r) {
    extern __shared__ __align__(16) float smem[];
    float *tile = smem;                       // [kTileRows][kWT]
    float *E = tile + kTileFloats;            // [kNB][2*NS][kWT]
    float *ER = E + kEFloats;                 // [2*NS][kWT]
    float *AGG = ER + kERFloats;              // [2*NS][kWT]; later 3 x kWT doubles

    cg::cluster_group cluster = cg::this_cluster();
    const int tid = threadIdx.x;
    const int R = cu.R;
    const int c0 = tx * p.Wout;               // first output channel of the tile
    const int cbase = c0 - p.HP;              // channel of tile column 0
    const int blk0 = r * cu.nbc;
    const int nb = min(cu.nbc, cu.nblk - blk0);   // blocks in this CTA (>= 1)
    const int row0 = blk0 * kL;               // first launch row of this CTA
    const int rows = min(nb * kL, cu.T - row0);
    const bool last_cta = (r == R - 1);
    if constexpr (DET) {
        // The long window's exiting cf values come from ring rows written at
        // least one launch ago: start their HBM -> L2 transfer now, behind the
        // IIR phases (one 128-byte line per thread; L2 is coherent, so a row
        // the previous launch is still writing is only fetched early).
        const int k = tid >> 1;
        if (k < rows && cu.n0 + row0 + k - p.nl >= 0) {
            const int slot = (int)((cu.n0 + row0 + k - p.nl) % cu.Q);
            const int cc = c0 + ((tid & 1) << 5);
            if (cc < cu.C) {
                const float *a = cu.ring + (long long)slot * cu.ldr + cc;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
            }
        }
    }

    // ---------------------------------------------------------------- 0. load
    {
        const float *xb = cu.x + (long long)row0 * cu.ldx;
        if (cu.x_vec4) {
#pragma unroll
            for (int it = 0; it < kTileFloats / 4 / kThreads; ++it) {
                const int f = tid + it * kThreads;
                const int row = f >> 4, col = (f & 15) << 2;
                const int cgl = cbase + col;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (row < rows) {
                    const float *src = xb + (long long)row * cu.ldx + cgl;
                    if (cgl >= 0 && cgl + 3 < cu.C) {
                        v = __ldg(reinterpret_cast<const float4 *>(src));
                    } else {
                        if (cgl + 0 >= 0 && cgl + 0 < cu.C) v.x = __ldg(src + 0);
                        if (cgl + 1 >= 0 && cgl + 1 < cu.C) v.y = __ldg(src + 1);
                        if (cgl + 2 >= 0 && cgl + 2 < cu.C) v.z = __ldg(src + 2);
                        if (cgl + 3 >= 0 && cgl + 3 < cu.C) v.w = __ldg(src + 3);
                    }
                }
                *reinterpret_cast<float4 *>(&tile[row * kWT + col]) = v;
            }
        } else {
            for (int f = tid; f < kTileFloats; f += kThreads) {
                const int row = f / kWT, col = f % kWT;
                const int cgl = cbase + col;
                float v = 0.f;
                if (row < rows && cgl >= 0 && cgl < cu.C) v = __ldg(xb + (long long)row * cu.ldx + cgl);
                tile[f] = v;
            }
        }
    }
    __syncthreads();

    // (channel, block) mapping: warps 2j, 2j+1 cover block j, columns 0-31 / 32-63
    const int warp = tid >> 5, lane = tid & 31;
    const int jb = warp >> 1;
    const int col = ((warp & 1) << 5) | lane;
    const int cgc = cbase + col;
    const bool col_owned = col >= p.HP && col < p.HP + p.Wout && cgc < cu.C;

    // ------------------------------------------------ 1. local responses
    if constexpr (NS > 0) {
        if (jb < nb) {
            const float *xc = tile + (jb * kL) * kWT + col;
            if (blk0 + jb == cu.nblk - 1 && cu.Lr < kL) {
                // ragged last block: its end state after Lr samples is K applied
                // to the input right-aligned in the block
                const int off = kL - cu.Lr;
                float e[2 * NS];
#pragma unroll
                for (int q = 0; q < 2 * NS; ++q) e[q] = 0.f;
#pragma unroll
                for (int i = 0; i < kL; ++i) {
                    const float xi = (i >= off) ? xc[(i - off) * kWT] : 0.f;
#pragma unroll
                    for (int q = 0; q < 2 * NS; ++q) e[q] = fmaf(p.tab.K[i][q], xi, e[q]);
                }
#pragma unroll
                for (int q = 0; q < 2 * NS; ++q) ER[q * kWT + col] = e[q];
            }
            float y[kL];
            float e[2 * NS];
#pragma unroll
            for (int k = 0; k < kL; ++k) y[k] = 0.f;
#pragma unroll
            for (int q = 0; q < 2 * NS; ++q) e[q] = 0.f;
#pragma unroll
            for (int i = 0; i < kL; ++i) {
                const float xi = xc[i * kWT];
#pragma unroll
                for (int k = i; k < kL; ++k) y[k] = fmaf(p.tab.h[k - i], xi, y[k]);
#pragma unroll
                for (int q = 0; q < 2 * NS; ++q) e[q] = fmaf(p.tab.K[i][q], xi, e[q]);
            }
#pragma unroll
            for (int q = 0; q < 2 * NS; ++q) E[(jb * 2 * NS + q) * kWT + col] = e[q];
            // the block's input is no longer needed: park y_loc in its place
            float *xw = tile + (jb * kL) * kWT + col;
#pragma unroll
            for (int k = 0; k < kL; ++k) xw[k * kWT] = y[k];
        }
    }

    // everything below reads state that the previous launch writes
    if (p.pdl) pdl_wait();
    __syncthreads();

    if constexpr (NS > 0) {
        // ------------------------------------------------ 2. carry scan
        if constexpr (DENSE) {
            // canonical basis, double-float carry at every block; lanes
            // 8k..8k+7 of warp v hold column 4v + k
            constexpr int n = 2 * NS;
            constexpr int kMat = kDenseDim * 8;                                   // float4 per matrix
            DF *AGGD = reinterpret_cast<DF *>(AGG);                               // [n][kWT]
            const int w = lane & 7, lane_base = lane & ~7;
            const int c = (warp << 2) | (lane >> 3);
            const bool act = w < NS;
            const int rlo = act ? w : 0, rhi = act ? n - 1 - w : 0;
            const int cgs = cbase + c;
            const bool ragged_last = last_cta && cu.Lr < kL;
            const float4 *Md = reinterpret_cast<const float4 *>(p.dense);
            const float4 *AL = Md + (kL - 1) * kMat;
            const float4 *Ar = Md + (cu.Lr - 1) * kMat;
            const float4 *Phi = Md + (kL + 1) * kMat;
            const float4 *PhiR = Md + (kL + r) * kMat;
            const DF zero{0.f, 0.f};
            DenseRows st{zero, zero};
            // (a) aggregate of this CTA from a zero start (not needed by the last)
            if (!last_cta) {
                for (int j = 0; j < nb; ++j) {
                    const DF al{act ? E[(j * n + rlo) * kWT + c] : 0.f, 0.f};
                    const DF ah{act ? E[(j * n + rhi) * kWT + c] : 0.f, 0.f};
                    dense_step<NS>(AL, st, al, ah, w, lane_base, p.all32);
                }
                if (act) {
                    AGGD[rlo * kWT + c] = st.lo;
                    AGGD[rhi * kWT + c] = st.hi;
                }
            }
            body_sync<SOLO>();
            // (b) g = sum over earlier CTAs q of Phi^(r-1-q) agg_q
            st = DenseRows{zero, zero};
            for (int q = 0; q < r; ++q) {
                const DF *ragg = cluster.map_shared_rank(AGGD, tile_rank(cluster, r, q));
                const DF al = act ? ragg[rlo * kWT + c] : zero;
                const DF ah = act ? ragg[rhi * kWT + c] : zero;
                dense_step<NS>(Phi, st, al, ah, w, lane_base, p.all32);
            }
            const DenseRows g = st;
            // (c) state at this CTA's start: Phi^r s_launch + g (FP64 in memory)
            {
                const double *src = cu.halo_in ? cu.halo_in + ((long long)tx * kWT + c) * n
                                               : cu.iir_in + (long long)cgs * n;
                const bool ok = act && cgs >= 0 && cgs < cu.C;
                st.lo = ok ? df_from_double(src[rlo]) : zero;
                st.hi = ok ? df_from_double(src[rhi]) : zero;
                dense_step<NS>(PhiR, st, g.lo, g.hi, w, lane_base, p.all32);
            }
            // (d) block start states (FP32 into E) and, in the last CTA, the end state
            for (int j = 0; j < nb; ++j) {
                const bool rag = ragged_last && j == nb - 1;
                DF al = zero, ah = zero;
                if (act) {
                    float *pl = &E[(j * n + rlo) * kWT + c], *ph = &E[(j * n + rhi) * kWT + c];
                    al.hi = rag ? ER[rlo * kWT + c] : *pl;
                    ah.hi = rag ? ER[rhi * kWT + c] : *ph;
                    *pl = st.lo.hi;
                    *ph = st.hi.hi;
                }
                if (last_cta || j < nb - 1) dense_step<NS>(rag ? Ar : AL, st, al, ah, w, lane_base, p.all32);
            }
            if (last_cta && act && cgs >= 0 && cgs < cu.C) {
                const double vlo = (double)st.lo.hi + (double)st.lo.lo;
                const double vhi = (double)st.hi.hi + (double)st.hi.lo;
                if (cu.iir_out && c >= p.HP && c < p.HP + p.Wout) {
                    cu.iir_out[(long long)cgs * n + rlo] = vlo;
                    cu.iir_out[(long long)cgs * n + rhi] = vhi;
                }
                if (cu.halo_out) {
                    cu.halo_out[((long long)tx * kWT + c) * n + rlo] = vlo;
                    cu.halo_out[((long long)tx * kWT + c) * n + rhi] = vhi;
                }
            }
        } else {
        const int sc = tid % kWT;
        constexpr int kSlotStep = kThreads / kWT;            // slots handled per pass
        const bool ragged_last = last_cta && cu.Lr < kL;
        // this CTA's aggregate per slot: end state of its range from a zero
        // start (FP32)
        for (int s = tid / kWT; s < NS; s += kSlotStep) {
            float a0 = 0.f, a1 = 0.f;
            for (int j = 0; j < nb; ++j) {
                float e0, e1, m00, m01, m10, m11;
                if (ragged_last && j == nb - 1) {
                    e0 = ER[(2 * s) * kWT + sc];
                    e1 = ER[(2 * s + 1) * kWT + sc];
                    m00 = cu.Mr32[s][0]; m01 = cu.Mr32[s][1]; m10 = cu.Mr32[s][2]; m11 = cu.Mr32[s][3];
                } else {
                    e0 = E[(j * 2 * NS + 2 * s) * kWT + sc];
                    e1 = E[(j * 2 * NS + 2 * s + 1) * kWT + sc];
                    m00 = p.tab.M[s][0]; m01 = p.tab.M[s][1]; m10 = p.tab.M[s][2]; m11 = p.tab.M[s][3];
                }
                const float t0 = fmaf(m00, a0, fmaf(m01, a1, e0));
                const float t1 = fmaf(m10, a0, fmaf(m11, a1, e1));
                a0 = t0;
                a1 = t1;
            }
            AGG[(2 * s) * kWT + sc] = a0;
            AGG[(2 * s + 1) * kWT + sc] = a1;
        }
        // publish the aggregates; meanwhile read the launch's carried state
        // (double-float hi/lo pairs) of this thread's slot
        static_assert(NS <= kSlotStep, "one slot per thread");
        body_arrive_release<SOLO>();
        float2 c0 = make_float2(0.f, 0.f), c1 = make_float2(0.f, 0.f);
        {
            const int s = tid / kWT, cgs = cbase + sc;
            if (s < NS && cgs >= 0 && cgs < cu.C) {
                const float2 *src = reinterpret_cast<const float2 *>(
                    cu.halo_in ? cu.halo_in + ((long long)tx * kWT + sc) * (2 * NS)
                               : cu.iir_in + (long long)cgs * (2 * NS));
                c0 = src[2 * s];
                c1 = src[2 * s + 1];
            }
        }
        body_wait<SOLO>();
        for (int s = tid / kWT; s < NS; s += kSlotStep) {
            const int cgs = cbase + sc;
            // earlier CTAs of the cluster: g = sum_q Phi^(r-1-q) agg_q, each
            // term from its own power (independent loads, FP32)
            float g0 = 0.f, g1 = 0.f;
            for (int q = 0; q < r; ++q) {
                const float *ragg = cluster.map_shared_rank(AGG, tile_rank(cluster, r, q));
                const float a0 = ragg[(2 * s) * kWT + sc], a1 = ragg[(2 * s + 1) * kWT + sc];
                const float *Pq = p.PhiPow32[r - 1 - q][s];
                g0 = fmaf(Pq[0], a0, fmaf(Pq[1], a1, g0));
                g1 = fmaf(Pq[2], a0, fmaf(Pq[3], a1, g1));
            }
            // the start of this CTA, Phi^r c + g, only feeds the FP32 block
            // carries
            const float *Pr = p.PhiPow32[r][s];
            const float d0 = fmaf(Pr[0], c0.x, fmaf(Pr[1], c1.x, g0));
            const float d1 = fmaf(Pr[2], c0.x, fmaf(Pr[3], c1.x, g1));
            const bool own = sc >= p.HP && sc < p.HP + p.Wout;
            if (last_cta && cgs >= 0 && cgs < cu.C && (own || cu.halo_out)) {
                // launch end state: PhiTot c + PhiLast g + own aggregate, in
                // double-float (~48 bits) on the FP32 pipe
                const float a0 = AGG[(2 * s) * kWT + sc], a1 = AGG[(2 * s + 1) * kWT + sc];
                const float *PTh = cu.PhiTotHi[s], *PTl = cu.PhiTotLo[s];
                const float *PLh = cu.PhiLastHi[s], *PLl = cu.PhiLastLo[s];
                const DF C0{c0.x, c0.y}, C1{c1.x, c1.y};
                DF u0 = df_add(df_add(df_mul(DF{PTh[0], PTl[0]}, C0), df_mul(DF{PTh[1], PTl[1]}, C1)),
                               df_add(df_add(df_mul_f(DF{PLh[0], PLl[0]}, g0), df_mul_f(DF{PLh[1], PLl[1]}, g1)),
                                      DF{a0, 0.f}));
                DF u1 = df_add(df_add(df_mul(DF{PTh[2], PTl[2]}, C0), df_mul(DF{PTh[3], PTl[3]}, C1)),
                               df_add(df_add(df_mul_f(DF{PLh[2], PLl[2]}, g0), df_mul_f(DF{PLh[3], PLl[3]}, g1)),
                                      DF{a1, 0.f}));
                if (p.all32) {
                    u0 = DF{u0.hi, 0.f};
                    u1 = DF{u1.hi, 0.f};
                }
                if (own && cu.iir_out) {
                    float2 *dst = reinterpret_cast<float2 *>(cu.iir_out + (long long)cgs * (2 * NS));
                    dst[2 * s] = make_float2(u0.hi, u0.lo);
                    dst[2 * s + 1] = make_float2(u1.hi, u1.lo);
                }
                if (cu.halo_out) {
                    float2 *dst = reinterpret_cast<float2 *>(cu.halo_out + ((long long)tx * kWT + sc) * (2 * NS));
                    dst[2 * s] = make_float2(u0.hi, u0.lo);
                    dst[2 * s + 1] = make_float2(u1.hi, u1.lo);
                }
            }
            // block start states (FP32), written over the block end states
            const float m00 = p.tab.M[s][0], m01 = p.tab.M[s][1], m10 = p.tab.M[s][2], m11 = p.tab.M[s][3];
            float f0 = d0, f1 = d1;
            for (int j = 0; j < nb; ++j) {
                float *pe0 = &E[(j * 2 * NS + 2 * s) * kWT + sc];
                float *pe1 = pe0 + kWT;
                const float e0 = *pe0, e1 = *pe1;
                *pe0 = f0;
                *pe1 = f1;
                const float t0 = fmaf(m00, f0, fmaf(m01, f1, e0));
                const float t1 = fmaf(m10, f0, fmaf(m11, f1, e1));
                f0 = t0;
                f1 = t1;
            }
        }
        }
        __syncthreads();

        // ------------------------------------------------ 3. fix-up
        if (jb < nb) {
            float m[2 * NS];
#pragma unroll
            for (int q = 0; q < 2 * NS; ++q) m[q] = E[(jb * 2 * NS + q) * kWT + col];
            float *tc = tile + (jb * kL) * kWT + col;
#pragma unroll
            for (int k = 0; k < kL; ++k) {
                float acc = tc[k * kWT];
#pragma unroll
                for (int q = 0; q < 2 * NS; ++q) acc = fmaf(p.tab.G[k][q], m[q], acc);
                tc[k * kWT] = acc;
            }
            if (cu.bp && col_owned) {
                float *bpc = cu.bp + (long long)(row0 + jb * kL) * cu.ldo + cgc;
                for (int k = 0; k < kL && jb * kL + k < rows; ++k) bpc[(long long)k * cu.ldo] = tc[k * kWT];
            }
        }
    } else {
        // no IIR stage: the bandpass output is the input
        if (cu.bp && col_owned && jb < nb) {
            for (int k = 0; k < kL; ++k) {
                const int row = jb * kL + k;
                if (row < rows) cu.bp[(long long)(row0 + row) * cu.ldo + cgc] = tile[row * kWT + col];
            }
        }
    }
    __syncthreads();

    // ------------------------------------------------ 4. spatial mean, cf
    // ring slot of tile row 0 (the host passes n0 mod Q; row0 < 2048 <= Q)
    int slot_r0 = cu.slot_n0 + row0;
    if (slot_r0 >= cu.Q) slot_r0 -= cu.Q;
    if (cu.sp || DET) {
        const int g = tid & 15, ro = tid >> 4;      // 4-column group, row offset (< kRowStep)
        const int ngroups = p.Wout >> 2;
        const int q0 = p.HP + 4 * g;                // first output column of the group
        const bool gact = g < ngroups;
        const int cch = c0 + 4 * g;
        // 1/|W| for the 4 channels (the window shrinks at the array ends)
        float inv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int lo = max(0, cch + u - p.hw), hi = min(cu.C - 1, cch + u + p.hw);
            inv[u] = 1.0f / (float)max(1, hi - lo + 1);
        }
        const bool full_group = cch + 3 < cu.C;
        // every thread takes the same branch (hw and HP are launch constants)
        switch (p.HP == 4 ? p.hw : (p.HP == 0 ? 0 : -1)) {
        case 0: spatial_rows<0, DET>(cu, tile, ro, rows, q0, row0, cch, slot_r0, full_group, gact, inv); break;
        case 1: spatial_rows<1, DET>(cu, tile, ro, rows, q0, row0, cch, slot_r0, full_group, gact, inv); break;
        case 2: spatial_rows<2, DET>(cu, tile, ro, rows, q0, row0, cch, slot_r0, full_group, gact, inv); break;
        case 3: spatial_rows<3, DET>(cu, tile, ro, rows, q0, row0, cch, slot_r0, full_group, gact, inv); break;
        case 4: spatial_rows<4, DET>(cu, tile, ro, rows, q0, row0, cch, slot_r0, full_group, gact, inv); break;
        default: spatial_rows_generic<DET>(p, cu, tile, ro, rows, q0, row0, cch, slot_r0, full_group, gact, inv); break;
        }
    }

    if constexpr (DET) {
        // ring writes of every CTA of the cluster become visible to the others
        // (release/acquire at cluster scope orders the global stores too; the
        // next launch sees them at the kernel boundary)
        body_sync<SOLO>();

        // ------------------------------------------------ 5. STA/LTA
        DF *DS = reinterpret_cast<DF *>(E + kDetDS);
        DF *DL = reinterpret_cast<DF *>(E + kDetDL);
        DF *BS = reinterpret_cast<DF *>(E + kDetBS);
        DF *BL = reinterpret_cast<DF *>(E + kDetBL);
        int *LZ = reinterpret_cast<int *>(E + kDetLZ);
        int *BZ = reinterpret_cast<int *>(E + kDetBZ);
        const bool dact = col_owned && jb < nb;
        const long long nrow0 = cu.n0 + row0;                 // global index of tile row 0
        const int rbeg = jb * kL;
        // The exiting values cf[n - w] of a block's 32 samples are read from
        // this tile when they all lie in it (mode 1), else from the history
        // ring, which phase 4 has already filled for this launch: as one
        // contiguous run (mode 0) or sample by sample with wrap-around and the
        // zeros before the first sample (mode 2).  Modes are warp-uniform.
        struct Exit {
            int mode, off, s0, lr0;
        };
        auto make_exit = [&](int w) -> Exit {
            Exit e;
            e.lr0 = rbeg - w;
            if (e.lr0 >= 0) {
                e.mode = 1;
                e.off = e.lr0 * kWT + col;
                e.s0 = 0;
                return e;
            }
            int slot = slot_r0 + e.lr0;          // > -Q
            if (slot < 0) slot += cu.Q;
            e.s0 = slot;
            e.off = slot * (int)cu.ldr + cgc;
            e.mode = (slot + kL - 1 < cu.Q && nrow0 + e.lr0 >= 0) ? 0 : 2;
            return e;
        };
        const Exit exS = make_exit(p.ns), exL = make_exit(p.nl);
        const int ldr = (int)cu.ldr;
        const bool full_blk = rbeg + kL <= rows;      // warp-uniform
        // eight exits starting at block sample kb (samples past `rows` read 0
        // unless the block is known to be full)
        auto fetch8 = [&](const Exit &e, int kb, float (&v)[8], auto full) {
            if (e.mode == 0) {
                const float *gp = cu.ring + (e.off + kb * ldr);
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = __ldcg(gp + u * ldr);
            } else if (e.mode == 1) {
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = tile[e.off + (kb + u) * kWT];
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    int slot = e.s0 + kb + u;
                    slot = slot >= cu.Q ? slot - cu.Q : slot;
                    const float t = __ldcg(cu.ring + (slot * ldr + cgc));
                    v[u] = (nrow0 + (e.lr0 + kb + u) >= 0) ? t : 0.f;
                }
            }
            if constexpr (!decltype(full)::value) {
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = (rbeg + kb + u < rows) ? v[u] : 0.f;
            }
        };
        // pass a: exact block sums of cf and of the exiting values (cf is 0 in
        // the tile past `rows`)
        auto pass_a = [&](auto full) {
            float cs = 0.f, cc = 0.f, ss = 0.f, sc2 = 0.f, ls = 0.f, lc = 0.f;
            int lz = kNoNonzero;
#pragma unroll 1
            for (int kb = 0; kb < kL; kb += 8) {
                float vs[8], vl[8];
                fetch8(exS, kb, vs, full);
                fetch8(exL, kb, vl, full);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float cf = tile[(rbeg + kb + u) * kWT + col];
                    acc_nonneg(cs, cc, cf);
                    acc_nonneg(ss, sc2, vs[u]);
                    acc_nonneg(ls, lc, vl[u]);
                    lz = cf != 0.f ? rbeg + kb + u : lz;
                }
            }
            const DF tot = df_from_sum(cs, cc);
            DS[jb * kWT + col] = df_add(tot, df_neg(df_from_sum(ss, sc2)));
            DL[jb * kWT + col] = df_add(tot, df_neg(df_from_sum(ls, lc)));
            LZ[jb * kWT + col] = lz;
        };
        if (dact) {
            if (full_blk) pass_a(std::true_type{});
            else pass_a(std::false_type{});
        }
        __syncthreads();
        // exclusive scan over this CTA's blocks, one thread per column
        // (double-float); AGG2 holds the CTA totals for the later CTAs:
        // [0..2) STA hi/lo, [2..4) LTA hi/lo, [4] 1 + last nonzero index (0 = none)
        float *AGG2 = AGG;                                   // [5][kWT]
        if (tid < kWT) {
            const int c = tid;
            const bool own = c >= p.HP && c < p.HP + p.Wout && cbase + c < cu.C;
            if (own) {
                DF bs{0.f, 0.f}, bl{0.f, 0.f};
                int bz = kNoNonzero;
                for (int j = 0; j < nb; ++j) {
                    BS[j * kWT + c] = bs;
                    BL[j * kWT + c] = bl;
                    BZ[j * kWT + c] = bz;
                    bs = df_add(bs, DS[j * kWT + c]);
                    bl = df_add(bl, DL[j * kWT + c]);
                    bz = max(bz, LZ[j * kWT + c]);
                }
                AGG2[0 * kWT + c] = bs.hi;
                AGG2[1 * kWT + c] = bs.lo;
                AGG2[2 * kWT + c] = bl.hi;
                AGG2[3 * kWT + c] = bl.lo;
                // the last nonzero as an index relative to the launch start
                AGG2[4 * kWT + c] = __int_as_float(bz == kNoNonzero ? kNoNonzero : row0 + bz);
            }
        }
        body_sync<SOLO>();
        if (tid < kWT) {
            const int c = tid;
            const int cgl = cbase + c;
            const bool own = c >= p.HP && c < p.HP + p.Wout && cgl < cu.C;
            if (own) {
                // state at the start of this CTA: carried state + earlier CTAs
                const double sIn = cu.det_in[(long long)cgl * 4 + 0];
                const double lIn = cu.det_in[(long long)cgl * 4 + 1];
                const double zIn = cu.det_in[(long long)cgl * 4 + 2];   // 1 + index of last nonzero, 0 = none
                DF bS{(float)sIn, 0.f}, bL{(float)lIn, 0.f};
                bS.lo = (float)(sIn - (double)bS.hi);
                bL.lo = (float)(lIn - (double)bL.hi);
                // last nonzero relative to the launch start (clamped)
                int zl = kNoNonzero;
                if (zIn > 0.0) {
                    const long long rel = (long long)zIn - 1 - cu.n0;
                    zl = rel < (long long)kNoNonzero ? kNoNonzero : (int)rel;
                }
                for (int q = 0; q < r; ++q) {
                    const float *ra = cluster.map_shared_rank(AGG2, tile_rank(cluster, r, q));
                    bS = df_add(bS, DF{ra[0 * kWT + c], ra[1 * kWT + c]});
                    bL = df_add(bL, DF{ra[2 * kWT + c], ra[3 * kWT + c]});
                    zl = max(zl, __float_as_int(ra[4 * kWT + c]));
                }
                if (last_cta) {
                    const DF eS = df_add(bS, DF{AGG2[0 * kWT + c], AGG2[1 * kWT + c]});
                    const DF eL = df_add(bL, DF{AGG2[2 * kWT + c], AGG2[3 * kWT + c]});
                    const int ez = max(zl, __float_as_int(AGG2[4 * kWT + c]));
                    cu.det_out[(long long)cgl * 4 + 0] = (double)eS.hi + (double)eS.lo;
                    cu.det_out[(long long)cgl * 4 + 1] = (double)eL.hi + (double)eL.lo;
                    cu.det_out[(long long)cgl * 4 + 2] = ez == kNoNonzero ? 0.0 : (double)(cu.n0 + ez + 1);
                    cu.det_out[(long long)cgl * 4 + 3] = 0.0;
                }
                // relative to this CTA's row 0
                const int bzr = zl == kNoNonzero ? kNoNonzero : zl - row0;
                for (int j = 0; j < nb; ++j) {
                    BS[j * kWT + c] = df_add(BS[j * kWT + c], bS);
                    BL[j * kWT + c] = df_add(BL[j * kWT + c], bL);
                    BZ[j * kWT + c] = max(BZ[j * kWT + c], bzr);
                }
            }
        }
        __syncthreads();
        // every read of another CTA's shared memory is done: the closing
        // cluster barrier's arrive (its wait is at the end of the body)
        body_arrive_relaxed<SOLO>();
        // pass b: running sums inside the block, ratio
        if (dact) {
            float fs = BS[jb * kWT + col].hi + BS[jb * kWT + col].lo;
            float fl = BL[jb * kWT + col].hi + BL[jb * kWT + col].lo;
            int lz = BZ[jb * kWT + col];
            // warm-up: rows before global index nl - 1 give 0
            const long long wl = (long long)(p.nl - 1) - nrow0;
            const int warm = wl > 4096 ? 4096 : (wl < -4096 ? -4096 : (int)wl);
            float *rp = cu.ratio ? cu.ratio + (long long)(row0 + rbeg) * cu.ldo + cgc : nullptr;
            const float scale = p.ratio_scale;
            // past the warm-up, with a nonzero cf inside every window of the
            // block already known, no sample needs the validity test
            const bool all_valid = full_blk && rbeg >= warm && lz > rbeg + kL - 1 - p.nl;
            TrigAuto ta;
            if (all_valid && rp) {
#pragma unroll 1
                for (int kb = 0; kb < kL; kb += 8) {
                    float vs[8], vl[8];
                    fetch8(exS, kb, vs, std::true_type{});
                    fetch8(exL, kb, vl, std::true_type{});
                    float *rq = rp + (long long)kb * cu.ldo;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const float cf = tile[(rbeg + kb + u) * kWT + col];
                        fs += cf - vs[u];
                        fl += cf - vl[u];
                        const float Rv = (fs * scale) * rcp_approx(fl);
                        rq[(long long)u * cu.ldo] = Rv;
                        if constexpr (TRIG) ta.step(Rv, p.trig_on, p.trig_off, kb + u);
                    }
                }
            } else {
#pragma unroll 1
                for (int kb = 0; kb < kL; kb += 8) {
                    float vs[8], vl[8];
                    fetch8(exS, kb, vs, std::false_type{});
                    fetch8(exL, kb, vl, std::false_type{});
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int row = rbeg + kb + u;
                        const float cf = tile[row * kWT + col];
                        fs += cf - vs[u];
                        fl += cf - vl[u];
                        lz = cf != 0.f ? row : lz;
                        const bool valid = (row >= warm) & (lz > row - p.nl);
                        const float Rv = valid ? (fs * scale) * rcp_approx(fl) : 0.f;
                        if (rp && row < rows) rp[(long long)(kb + u) * cu.ldo] = Rv;
                        if constexpr (TRIG)
                            if (row < rows) ta.step(Rv, p.trig_on, p.trig_off, kb + u);
                    }
                }
            }
            if constexpr (TRIG) cu.trig_summ[(long long)(blk0 + jb) * cu.C + cgc] = ta.packed();
        }
    }
    // no CTA may exit while a peer can still read its shared memory
    if constexpr (DET) body_wait<SOLO>();
    else if (NS > 0) body_sync<SOLO>();
}

template <int NS, bool DET>
__host__ __device__ constexpr int chain_cluster_barriers() {
    return (NS > 0 ? 1 : 0) + (DET ? 2 : 0) + ((NS > 0 || DET) ? 1 : 0);
}

}  // namespace
}  // namespace filark
