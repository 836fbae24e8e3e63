// Differentiable SOS cascade: a forward pass that keeps the cascade state at
// checkpoints, and the reverse-time adjoint that gives the gradients with
// respect to the input and to all six coefficients of every section, so the
// bandpass of the chain can be fitted or inverted.
//
// Section s maps u_s -> y_s = u_{s+1} by
//     a0 y[n] + a1 y[n-1] + a2 y[n-2] = b0 u[n] + b1 u[n-1] + b2 u[n-2]
// from zero state, evaluated in transposed direct form II with the
// coefficients divided by a0 (Sec. 3.4, the SOS filter).  For a loss L with
// g = dL/dy_{S-1}, the adjoint w_s of section s solves, backwards in time,
//     a0 w[n] + a1 w[n+1] + a2 w[n+2] = g_s[n],   w = 0 after the last sample,
// and
//     dL/db_i  =  sum_m u_s[m] w_s[m+i],
//     dL/da_i  = -sum_m y_s[m] w_s[m+i],
//     g_{s-1}[n] = dL/du_s[n] = b0 w_s[n] + b1 w_s[n+1] + b2 w_s[n+2].
//
// Arithmetic is double-float (FP32 pairs, ~48 significant bits) on the FP32
// pipe -- GB300 runs FP64 at 1/64 of the FP32 rate.  Plain FP32 is not enough:
// for poles a few 1e-3 from z = 1, rounding the coefficients alone moves the
// poles by ~1e-5 and the resonance gain by ~1e-3.  Only the final reduction of
// the coefficient gradients runs in FP64.
//
// Parallelism over time as well as channels.  The record is cut into segments
// of at most `ckpt` samples; one thread owns one (segment, channel) pair.  When
// the channels times the segments of `ckpt` samples are too few threads to
// fill the GPU (kTargetThreads), the segments are shortened (to no fewer than
// kMinSegment samples) until they are enough: the checkpoints are then closer
// than asked for, which the size queries account for.  Both the forward state
// and the adjoint state are linear in their inputs, so each pass runs in three
// steps: every thread forms the state its segment ends in from a zero start
// (in block form, local_block_kernel); one group of lanes per channel chains
// the segments, state_next = T * state + local (T = the transition over a
// segment of zero input, computed on the host in long double); every thread
// reruns its segment from the true state.
//
// Memory: the forward's rerun keeps the cascade state at the start of every
// piece of P ~ sqrt(2 ckpt) samples (the checkpoints).  The backward
// recomputes a segment's section signals piece by piece, last to first, from
// those states into a P-sample buffer and consumes them in the adjoint.  The
// workspace holds (2S + P * S + 6S) doubles per (segment, channel) -- adjoint
// states, one piece of section signals, gradient partials -- instead of
// ckpt * S.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "filark_internal.h"
#include "host_trace.h"

namespace {

using filark::set_last_error;

constexpr int kMaxS = FILARK_MAX_SECTIONS;
constexpr int kMaxState = 2 * kMaxS;
constexpr int kAdjThreads = 128;
constexpr long long kTargetThreads = 1LL << 17;   // (segment, channel) pairs that fill the GPU
constexpr long long kMinSegment = 128;
constexpr int kChainThreads = 64;   // small CTAs: the chaining has only C x (2S rounded up) threads

// A double-float number (hi + lo, ~48 significant bits) on the FP32 pipe.
// The recursions are sums of products, so their one primitive is a fused
// acc + a * b: the leading product split exactly (TwoProduct by FMA), added
// to acc.hi exactly (Knuth's TwoSum), the rounding errors and the cross terms
// a.hi * b.lo, a.lo * b.hi gathered in the low word (as in the compensated dot
// product of Ogita, Rump and Oishi, 2005).  The sum is left unnormalised
// between the terms of one expression and renormalised (Dekker's Fast2Sum)
// once per value the recursion keeps.  Explicit-rounding intrinsics keep the
// compiler from contracting the error-free steps into FMAs.
struct dd {
    float hi, lo;
};
__device__ __forceinline__ dd dd_norm(float s, float e) {
    const float hi = __fadd_rn(s, e);
    return dd{hi, __fsub_rn(e, __fsub_rn(hi, s))};
}
__device__ __forceinline__ dd dd_renorm(dd v) { return dd_norm(v.hi, v.lo); }
__device__ __forceinline__ dd operator-(dd a) { return dd{-a.hi, -a.lo}; }
// a * b, unnormalised
__device__ __forceinline__ dd dd_mul_raw(dd a, dd b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return dd{p, e};
}
// acc + a * b, unnormalised (acc may be unnormalised too)
__device__ __forceinline__ dd dd_fma(dd acc, dd a, dd b) {
    const dd m = dd_mul_raw(a, b);
    const float s = __fadd_rn(acc.hi, m.hi);
    const float bb = __fsub_rn(s, acc.hi);
    const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(m.hi, bb));
    return dd{s, __fadd_rn(acc.lo, __fadd_rn(err, m.lo))};
}
__device__ __forceinline__ dd dd_f(float v) { return dd{v, 0.f}; }
__device__ __forceinline__ float dd_to_f(dd v) { return v.hi + v.lo; }
// storage: a double-float in an 8-byte slot of the double-typed buffers
__device__ __forceinline__ dd ld_dd(const double *p) {
    const float2 v = *reinterpret_cast<const float2 *>(p);
    return dd{v.x, v.y};
}
__device__ __forceinline__ void st_dd(double *p, dd v) { *reinterpret_cast<float2 *>(p) = make_float2(v.hi, v.lo); }

struct DDC {
    float hi, lo;
};

struct SosCoef {
    double b[kMaxS][3];   // numerators as given
    double a[kMaxS][3];   // denominators as given (a0 included)
    double nb[kMaxS][3];  // b / a0
    double na[kMaxS][2];  // a1 / a0, a2 / a0
    double ia0[kMaxS];    // 1 / a0
    // the same as double-float pairs for the kernels
    DDC db[kMaxS][3], da[kMaxS][3], dnb[kMaxS][3], dna[kMaxS][2], dia0[kMaxS];
};

struct Transition {
    double T[kMaxState][kMaxState];  // row-major, first 2S x 2S used
};

// Block form of the local passes: over a block of kLocalL samples the state
// (zero-input step A, e = the state one step after a unit input from a zero
// state) moves as z <- A^L z + sum_m K[m] u[m] with K[m] = A^(L-1-m) e.
constexpr int kLocalL = 64;
struct LocalTables {
    DDC AL[kMaxState][kMaxState];  // A^L, first D x D used
    DDC K[kLocalL][kMaxState];     // K[m][i], first D columns used
};

struct Geometry {
    long long N, ckpt, P;  // samples, segment length (<= the requested interval), piece length
    long long nseg, npiece;
    int C;
    long long NT;  // nseg * C threads
};

// ---- forward recursion (one TDF-II step of section s) ----------------------

template <typename R>
__host__ __device__ __forceinline__ R tdf2_step(const SosCoef &k, int s, R u, R &z1, R &z2) {
    const R y = (R)k.nb[s][0] * u + z1;
    z1 = (R)k.nb[s][1] * u - (R)k.na[s][0] * y + z2;
    z2 = (R)k.nb[s][2] * u - (R)k.na[s][1] * y;
    return y;
}

// ---- adjoint recursion (one reverse-time step of section s) ----------------
// w1 = w[n+1], w2 = w[n+2] on entry; returns g_{s-1}[n] and shifts the state.

template <typename R>
__host__ __device__ __forceinline__ R adj_step(const SosCoef &k, int s, R g, R &w1, R &w2, R &w) {
    w = (g - (R)k.a[s][1] * w1 - (R)k.a[s][2] * w2) * (R)k.ia0[s];
    const R gprev = (R)k.b[s][0] * w + (R)k.b[s][1] * w1 + (R)k.b[s][2] * w2;
    w2 = w1;
    w1 = w;
    return gprev;
}

__device__ __forceinline__ dd cf(const DDC &c) { return dd{c.hi, c.lo}; }

// tdf2_step in double-float: three fused sums of products, each renormalised
// once (y, and the two states the next step reads).
__device__ __forceinline__ dd tdf2_dd(const SosCoef &k, int s, dd u, dd &z1, dd &z2) {
    const dd y = dd_renorm(dd_fma(z1, cf(k.dnb[s][0]), u));
    z1 = dd_renorm(dd_fma(dd_fma(z2, cf(k.dnb[s][1]), u), -cf(k.dna[s][0]), y));
    z2 = dd_renorm(dd_fma(dd_mul_raw(cf(k.dnb[s][2]), u), -cf(k.dna[s][1]), y));
    return y;
}

// adj_step in double-float, with the denominator divided through:
// w = g / a0 - (a1 / a0) w1 - (a2 / a0) w2.  The value passed down the
// sections (g, then w) enters each sum last: the terms of the state are
// summed while it is still on its way.
__device__ __forceinline__ dd adj_dd(const SosCoef &k, int s, dd g, dd &w1, dd &w2, dd &w) {
    w = dd_renorm(dd_fma(dd_fma(dd_mul_raw(-cf(k.dna[s][0]), w1), -cf(k.dna[s][1]), w2), cf(k.dia0[s]), g));
    const dd gprev =
        dd_renorm(dd_fma(dd_fma(dd_mul_raw(cf(k.db[s][1]), w1), cf(k.db[s][2]), w2), cf(k.db[s][0]), w));
    w2 = w1;
    w1 = w;
    return gprev;
}

__device__ __forceinline__ void seg_range(const Geometry &g, long long seg, long long &t0, long long &t1) {
    t0 = seg * g.ckpt;
    t1 = t0 + g.ckpt < g.N ? t0 + g.ckpt : g.N;
}

// State and signal buffers are [row][NT] with the thread index fastest
// (coalesced); each 8-byte entry holds a double-float.
__device__ __forceinline__ long long ix(long long row, long long NT, long long T) { return row * NT + T; }

// acc + a * v for a double-float a and a float v, unnormalised
__device__ __forceinline__ dd dd_fma_f(dd acc, const DDC &a, float v) {
    const float p = __fmul_rn(a.hi, v);
    float e = fmaf(a.hi, v, -p);
    e = fmaf(a.lo, v, e);
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    return dd{s, __fadd_rn(acc.lo, __fadd_rn(err, e))};
}

// F1 / B1: the state each segment ends in from a zero start (the forward:
// every segment but the last, stored in the checkpoint slot of the next one;
// the adjoint, which runs backwards in time: every segment but the first, its
// adjoint state (w_s[n+1], w_s[n+2]) at the segment start stored in the slot of
// the previous one).  From a zero start that state is linear in the segment's
// input, so it is formed block by block from the tables (z <- A^L z +
// sum_m K[m] u[m]): D + D^2 / L double-float products per sample instead of the
// S sections' recursions.  Samples are taken in the recursion's order (the
// adjoint from the segment's end); the first block is the partial one, its
// len mod L samples at positions L - r .. L - 1.
template <int S, bool ADJ>
__global__ void __launch_bounds__(kAdjThreads) local_block_kernel(const __grid_constant__ LocalTables tb,
                                                                  const __grid_constant__ Geometry g,
                                                                  const float *__restrict__ in, long long ld,
                                                                  double *__restrict__ out) {
    constexpr int D = 2 * S;
    // K in shared memory, row m as D / 2 float4 (two double-float entries
    // each): every thread reads the same row, a broadcast
    __shared__ float4 sK[kLocalL][D / 2];
    for (int e = threadIdx.x; e < kLocalL * (D / 2); e += blockDim.x) {
        const int m = e / (D / 2), i = 2 * (e % (D / 2));
        sK[m][i / 2] = make_float4(tb.K[m][i].hi, tb.K[m][i].lo, tb.K[m][i + 1].hi, tb.K[m][i + 1].lo);
    }
    __syncthreads();
    const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (T >= g.NT) return;
    const long long seg = T / g.C;
    const int c = (int)(T - seg * g.C);
    if (ADJ ? seg == 0 : seg == g.nseg - 1) return;
    long long t0, t1;
    seg_range(g, seg, t0, t1);
    const long long len = t1 - t0;
    // acc[i] += K[m][i] v for all i
    auto add_sample = [&](dd(&acc)[D], int m, float v) {
#pragma unroll
        for (int h = 0; h < D / 2; ++h) {
            const float4 k2 = sK[m][h];
            acc[2 * h] = dd_fma_f(acc[2 * h], DDC{k2.x, k2.y}, v);
            acc[2 * h + 1] = dd_fma_f(acc[2 * h + 1], DDC{k2.z, k2.w}, v);
        }
    };
    // sample q of the recursion's order
    const float *src = in + (ADJ ? (t1 - 1) * ld : t0 * ld) + c;
    const long long step = ADJ ? -ld : ld;
    dd z[D];
#pragma unroll
    for (int i = 0; i < D; ++i) z[i] = dd_f(0.f);
    long long q = 0;
    const int r = (int)(len % kLocalL);
    if (r) {
        dd acc[D];
#pragma unroll
        for (int i = 0; i < D; ++i) acc[i] = dd_f(0.f);
        for (int m = kLocalL - r; m < kLocalL; ++m, ++q) add_sample(acc, m, src[q * step]);
#pragma unroll
        for (int i = 0; i < D; ++i) z[i] = dd_renorm(acc[i]);
    }
    for (; q < len; q += kLocalL) {
        dd acc[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            acc[i] = dd_mul_raw(cf(tb.AL[i][0]), z[0]);
#pragma unroll
            for (int j = 1; j < D; ++j) acc[i] = dd_fma(acc[i], cf(tb.AL[i][j]), z[j]);
        }
        const float *blk = src + q * step;
#pragma unroll 8
        for (int m = 0; m < kLocalL; ++m) add_sample(acc, m, blk[m * step]);
#pragma unroll
        for (int i = 0; i < D; ++i) z[i] = dd_renorm(acc[i]);
    }
    const long long To = ADJ ? T - g.C : T + g.C;
#pragma unroll
    for (int i = 0; i < D; ++i) st_dd(out + ix(i, g.NT, To), z[i]);
}

// F2 / B2: per channel, chain the segments (one D x D product per segment,
// double-float on the FP32 pipe).  A group of G >= D lanes serves one channel,
// lane i owning state row i; the state vector is read across the group with
// shuffles.
//   forward : st[0] = 0,         st[j+1] += T st[j]        (j ascending)
//   backward: st[nseg-1] = 0,    st[j-1] += T st[j]        (j descending)
template <int S>
__host__ __device__ constexpr int chain_group() {
    return 2 * S <= 2 ? 2 : (2 * S <= 4 ? 4 : (2 * S <= 8 ? 8 : 16));
}

// a + b for unnormalised double-float a, b (TwoSum of the leading words)
__device__ __forceinline__ dd dd_add_raw(dd a, dd b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return dd{s, __fadd_rn(__fadd_rn(a.lo, b.lo), err)};
}

// asynchronous 8-byte global -> shared copies (cp.async), own copies only
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The local states of kChainStage steps are copied into the thread's own
// column of a shared-memory stage while the previous kChainStage steps are
// combined (double-buffered), so the loads of a whole stage are in flight
// together instead of one step ahead.
constexpr int kChainStage = 32;

template <int S>
__global__ void __launch_bounds__(kChainThreads) chain_segments_kernel(const __grid_constant__ Transition tr,
                                                                       const __grid_constant__ Geometry g,
                                                                       double *__restrict__ st, int backward) {
    constexpr int D = 2 * S;
    constexpr int G = chain_group<S>();
    __shared__ float2 stage[2][kChainStage][kChainThreads];
    const int i = threadIdx.x % G;                          // state row of this lane
    const int gbase = (threadIdx.x & 31) - i;                // first lane of the group
    const long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const bool row = c < g.C && i < D;                       // lanes past D or C only shuffle
    dd Trow[D];
#pragma unroll
    for (int q = 0; q < D; ++q) {
        const double t = i < D ? tr.T[i][q] : 0.0;
        const float hi = (float)t;
        Trow[q] = dd{hi, (float)(t - (double)hi)};
    }
    dd v = dd_f(0.f);
    const long long first = backward ? g.nseg - 1 : 0;
    if (row) st_dd(st + ix(i, g.NT, first * g.C + c), dd_f(0.f));
    // steps j0 .. j0 + kChainStage - 1 (those < nseg) into stage[buf]
    auto issue = [&](int buf, long long j0) {
        if (row)
            for (int q = 0; q < kChainStage && j0 + q < g.nseg; ++q) {
                const long long seg = backward ? g.nseg - 1 - (j0 + q) : j0 + q;
                cp_async8(&stage[buf][q][threadIdx.x], st + ix(i, g.NT, seg * g.C + c));
            }
        cp_async_commit();
    };
    issue(0, 1);
    for (long long j0 = 1, sb = 0; j0 < g.nseg; j0 += kChainStage, sb ^= 1) {
        issue((int)sb ^ 1, j0 + kChainStage);
        cp_async_wait<1>();  // this thread's copies of stage sb have landed
        const int nq = g.nseg - j0 < kChainStage ? (int)(g.nseg - j0) : kChainStage;
        for (int q = 0; q < nq; ++q) {
            const long long j = j0 + q;
            const long long seg = backward ? g.nseg - 1 - j : j;
            const float2 lv = stage[sb][q][threadIdx.x];
            // two interleaved sums halve the dependent chain
            dd acc0 = row ? dd{lv.x, lv.y} : dd_f(0.f), acc1 = dd_f(0.f);
#pragma unroll
            for (int r = 0; r < D; ++r) {
                const dd vr{__shfl_sync(0xffffffffu, v.hi, gbase + r), __shfl_sync(0xffffffffu, v.lo, gbase + r)};
                if (r & 1)
                    acc1 = dd_fma(acc1, Trow[r], vr);
                else
                    acc0 = dd_fma(acc0, Trow[r], vr);
            }
            const dd acc = dd_renorm(dd_add_raw(acc0, acc1));
            v = row ? acc : dd_f(0.f);
            if (row) st_dd(st + ix(i, g.NT, seg * g.C + c), acc);
        }
    }
    cp_async_wait<0>();
}

// F3: rerun every segment from its checkpoint, writing y (if asked for) and
// the state at the start of every later piece of P samples (the pieces the
// backward recomputes one at a time), checkpoint rows p * 2S + r.
template <int S>
__global__ void __launch_bounds__(kAdjThreads) fwd_run_kernel(const __grid_constant__ SosCoef k,
                                                              const __grid_constant__ Geometry g,
                                                              const float *__restrict__ x, long long ldx,
                                                              double *__restrict__ ckpt,
                                                              float *__restrict__ y, long long ldy) {
    const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (T >= g.NT) return;
    const long long seg = T / g.C;
    const int c = (int)(T - seg * g.C);
    long long t0, t1;
    seg_range(g, seg, t0, t1);
    dd z[S][2];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        z[s][0] = ld_dd(ckpt + ix(2 * s, g.NT, T));
        z[s][1] = ld_dd(ckpt + ix(2 * s + 1, g.NT, T));
    }
    long long next = t0 + g.P, p = 1;
    float xn = x[t0 * ldx + c];  // loaded one sample ahead
    for (long long n = t0; n < t1; ++n) {
        if (n == next) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                st_dd(ckpt + ix(p * (2 * S) + 2 * s, g.NT, T), z[s][0]);
                st_dd(ckpt + ix(p * (2 * S) + 2 * s + 1, g.NT, T), z[s][1]);
            }
            ++p;
            next += g.P;
        }
        dd u = dd_f(xn);
        if (n + 1 < t1) xn = x[(n + 1) * ldx + c];
#pragma unroll
        for (int s = 0; s < S; ++s) u = tdf2_dd(k, s, u, z[s][0], z[s][1]);
        if (y) y[n * ldy + c] = dd_to_f(u);
    }
}

// acc += a * b for double-float a, b, the accumulator kept unnormalised
// over the whole run (its low word gathers every rounding error and cross
// term).
__device__ __forceinline__ void dd_acc_mul(dd &acc, dd a, dd b) { acc = dd_fma(acc, a, b); }

// B3: gradients.  The pieces (the forward left the state at each piece start
// in the checkpoints) are handled last to first: recompute the piece's
// section outputs into `sig` ([p][s][NT]), run the adjoint over it backwards
// from the true adjoint state, accumulate the coefficient gradients, write
// dL/dx.
template <int S>
__global__ void __launch_bounds__(kAdjThreads) adj_run_kernel(const __grid_constant__ SosCoef k,
                                                              const __grid_constant__ Geometry g,
                                                              const float *__restrict__ x, long long ldx,
                                                              const float *__restrict__ gy, long long ldg,
                                                              const double *__restrict__ ckpt,
                                                              const double *__restrict__ beta,
                                                              double *__restrict__ sig,
                                                              float *__restrict__ gx, long long ldgx,
                                                              double *__restrict__ gpart) {
    const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (T >= g.NT) return;
    const long long seg = T / g.C;
    const int c = (int)(T - seg * g.C);
    const long long NT = g.NT;
    long long t0, t1;
    seg_range(g, seg, t0, t1);
    const long long npiece = (t1 - t0 + g.P - 1) / g.P;

    dd w1[S], w2[S], gb[S][3], ga[S][3];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        w1[s] = ld_dd(beta + ix(2 * s, NT, T));
        w2[s] = ld_dd(beta + ix(2 * s + 1, NT, T));
#pragma unroll
        for (int i = 0; i < 3; ++i) gb[s][i] = ga[s][i] = dd_f(0.f);
    }
    for (long long p = npiece - 1; p >= 0; --p) {
        const long long a = t0 + p * g.P;
        const long long b = a + g.P < t1 ? a + g.P : t1;
        {
            dd z[S][2];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                z[s][0] = ld_dd(ckpt + ix(p * (2 * S) + 2 * s, NT, T));
                z[s][1] = ld_dd(ckpt + ix(p * (2 * S) + 2 * s + 1, NT, T));
            }
            float xn = x[a * ldx + c];  // loaded one sample ahead
            for (long long n = a; n < b; ++n) {
                dd u = dd_f(xn);
                if (n + 1 < b) xn = x[(n + 1) * ldx + c];
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    u = tdf2_dd(k, s, u, z[s][0], z[s][1]);
                    st_dd(sig + ix((n - a) * S + s, NT, T), u);
                }
            }
        }
        // the loads of sample n (y_s for every section, x, dL/dy) are issued
        // one sample ahead
        float gyn = gy[(b - 1) * ldg + c], xn = x[(b - 1) * ldx + c];
        dd sn[S];
#pragma unroll
        for (int s = 0; s < S; ++s) sn[s] = ld_dd(sig + ix((b - 1 - a) * S + s, NT, T));
        for (long long n = b - 1; n >= a; --n) {
            dd gg = dd_f(gyn);
            const float xc = xn;
            dd yv[S];
#pragma unroll
            for (int s = 0; s < S; ++s) yv[s] = sn[s];
            if (n > a) {
                gyn = gy[(n - 1) * ldg + c];
                xn = x[(n - 1) * ldx + c];
#pragma unroll
                for (int s = 0; s < S; ++s) sn[s] = ld_dd(sig + ix((n - 1 - a) * S + s, NT, T));
            }
            dd ys = yv[S - 1];
#pragma unroll
            for (int s = S - 1; s >= 0; --s) {
                // section s maps u_s = y_{s-1} (x for s = 0) to y_s
                const dd us = s == 0 ? dd_f(xc) : yv[s - 1];
                const dd wn1 = w1[s], wn2 = w2[s];
                dd w;
                gg = adj_dd(k, s, gg, w1[s], w2[s], w);
                dd_acc_mul(gb[s][0], us, w);
                dd_acc_mul(gb[s][1], us, wn1);
                dd_acc_mul(gb[s][2], us, wn2);
                // ga[s][0] (dL/da0) follows from the other five after the
                // reduction (finish_a0_kernel)
                dd_acc_mul(ga[s][1], ys, wn1);     // negated at the end
                dd_acc_mul(ga[s][2], ys, wn2);
                ys = us;
            }
            if (gx) gx[n * ldgx + c] = dd_to_f(gg);
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gpart[ix(6 * s + i, NT, T)] = (double)gb[s][i].hi + (double)gb[s][i].lo;
            gpart[ix(6 * s + 3 + i, NT, T)] = i == 0 ? 0.0 : -((double)ga[s][i].hi + (double)ga[s][i].lo);
        }
}

// B4: dL/dsos[j] = sum over all (segment, channel) partials, FP64, in a fixed
// order, by two launches of this kernel: CTA (j, q) sums chunk q of the n
// entries of row j (each thread 4 interleaved sums, combined in a fixed tree)
// into out[j * gridDim.y + q]; the second launch sums each row's chunk sums.
constexpr int kSumThreads = 1024;
constexpr int kSumSplit = 8;  // chunks per row in the first launch: 6 S x 8 CTAs
__global__ void __launch_bounds__(kSumThreads) sum_rows_kernel(const double *__restrict__ in, long long n,
                                                               long long ld, double *__restrict__ out) {
    __shared__ double part[kSumThreads];
    const int j = blockIdx.x, q = blockIdx.y, nq = gridDim.y;
    const long long chunk = (n + nq - 1) / nq;
    const long long lo = (long long)q * chunk;
    const long long len = lo < n ? (n - lo < chunk ? n - lo : chunk) : 0;
    const double *src = in + (long long)j * ld + lo;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    long long t = threadIdx.x;
    for (; t + 3 * kSumThreads < len; t += 4 * kSumThreads) {
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] += src[t + r * kSumThreads];
    }
    for (int r = 0; r < 4; ++r, t += kSumThreads)
        if (t < len) acc[r] += src[t];
    part[threadIdx.x] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    __syncthreads();
    for (int w = kSumThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[(long long)j * nq + q] = part[0];
}

// B5: dL/da0 of each section.  Scaling a section's six coefficients by the
// same factor leaves the cascade unchanged, so the loss is homogeneous of
// degree 0 in them and (Euler) sum_k c_k dL/dc_k = 0: dL/da0 =
// -(b0 gb0 + b1 gb1 + b2 gb2 + a1 ga1 + a2 ga2) / a0, from the reduced FP64
// sums -- one product per section and sample fewer in adj_run.
__global__ void finish_a0_kernel(const __grid_constant__ SosCoef k, int S, double *__restrict__ gsos) {
    const int s = threadIdx.x;
    if (s >= S) return;
    double *g = gsos + 6 * s;
    const double acc = k.b[s][0] * g[0] + k.b[s][1] * g[1] + k.b[s][2] * g[2] + k.a[s][1] * g[4] + k.a[s][2] * g[5];
    g[3] = -acc / k.a[s][0];
}

// ---- host side ---------------------------------------------------------------

bool load_coef(const double *sos, int S, SosCoef &k) {
    std::memset(&k, 0, sizeof(k));
    for (int s = 0; s < S; ++s) {
        const double *r = sos + 6 * s;
        for (int i = 0; i < 6; ++i)
            if (!std::isfinite(r[i])) return false;
        if (r[3] == 0.0) return false;
        for (int i = 0; i < 3; ++i) {
            k.b[s][i] = r[i];
            k.a[s][i] = r[3 + i];
            k.nb[s][i] = r[i] / r[3];
        }
        k.na[s][0] = r[4] / r[3];
        k.na[s][1] = r[5] / r[3];
        k.ia0[s] = 1.0 / r[3];
        auto split = [](double v) {
            DDC d;
            d.hi = (float)v;
            d.lo = (float)(v - (double)d.hi);
            return d;
        };
        for (int i = 0; i < 3; ++i) {
            k.db[s][i] = split(k.b[s][i]);
            k.da[s][i] = split(k.a[s][i]);
            k.dnb[s][i] = split(k.nb[s][i]);
        }
        k.dna[s][0] = split(k.na[s][0]);
        k.dna[s][1] = split(k.na[s][1]);
        k.dia0[s] = split(k.ia0[s]);
    }
    return true;
}

// The kernels' own zero-input recursions, one step, in long double: column q
// of the one-step matrix is the step applied to unit vector q.
void one_step_matrix(const SosCoef &k, int S, bool adjoint, long double M[kMaxState][kMaxState]) {
    const int D = 2 * S;
    for (int q = 0; q < D; ++q) {
        long double v[kMaxState] = {};
        v[q] = 1.0L;
        if (!adjoint) {
            long double u = 0.0L;
            for (int s = 0; s < S; ++s) u = tdf2_step<long double>(k, s, u, v[2 * s], v[2 * s + 1]);
        } else {
            long double gg = 0.0L, w;
            for (int s = S - 1; s >= 0; --s) gg = adj_step<long double>(k, s, gg, v[2 * s], v[2 * s + 1], w);
        }
        for (int i = 0; i < D; ++i) M[i][q] = v[i];
    }
}

void mat_mul(int D, const long double A[kMaxState][kMaxState], const long double B[kMaxState][kMaxState],
             long double R[kMaxState][kMaxState]) {
    long double t[kMaxState][kMaxState];
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            long double acc = 0.0L;
            for (int q = 0; q < D; ++q) acc += A[i][q] * B[q][j];
            t[i][j] = acc;
        }
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) R[i][j] = t[i][j];
}

// transition over n steps of zero input, by repeated squaring
void transition(const SosCoef &k, int S, bool adjoint, long long n, Transition &out) {
    const int D = 2 * S;
    long double M[kMaxState][kMaxState], R[kMaxState][kMaxState];
    one_step_matrix(k, S, adjoint, M);
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) R[i][j] = i == j ? 1.0L : 0.0L;
    while (n > 0) {
        if (n & 1) mat_mul(D, R, M, R);
        n >>= 1;
        if (n) mat_mul(D, M, M, M);
    }
    std::memset(&out, 0, sizeof(out));
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) out.T[i][j] = (double)R[i][j];
}

// The local passes' tables (A^L and K[m] = A^(L-1-m) e) from the kernels' own
// one-step recursion, in long double, split into double-float pairs.
void local_tables(const SosCoef &k, int S, bool adjoint, LocalTables &tb) {
    const int D = 2 * S;
    long double A[kMaxState][kMaxState], AL[kMaxState][kMaxState];
    one_step_matrix(k, S, adjoint, A);
    long double e[kMaxState] = {};
    if (!adjoint) {
        long double u = 1.0L;
        for (int s = 0; s < S; ++s) u = tdf2_step<long double>(k, s, u, e[2 * s], e[2 * s + 1]);
    } else {
        long double gg = 1.0L, w;
        for (int s = S - 1; s >= 0; --s) gg = adj_step<long double>(k, s, gg, e[2 * s], e[2 * s + 1], w);
    }
    long double K[kLocalL][kMaxState] = {};
    for (int i = 0; i < D; ++i) K[kLocalL - 1][i] = e[i];
    for (int m = kLocalL - 2; m >= 0; --m)
        for (int i = 0; i < D; ++i) {
            long double acc = 0.0L;
            for (int j = 0; j < D; ++j) acc += A[i][j] * K[m + 1][j];
            K[m][i] = acc;
        }
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) AL[i][j] = A[i][j];
    for (int n = 1; n < kLocalL; n *= 2) mat_mul(D, AL, AL, AL);  // kLocalL is a power of two
    auto split = [](long double v) {
        DDC d;
        d.hi = (float)v;
        d.lo = (float)(v - (long double)d.hi);
        return d;
    };
    std::memset(&tb, 0, sizeof(tb));
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) tb.AL[i][j] = split(AL[i][j]);
    for (int m = 0; m < kLocalL; ++m)
        for (int i = 0; i < D; ++i) tb.K[m][i] = split(K[m][i]);
}
static_assert((kLocalL & (kLocalL - 1)) == 0, "kLocalL: a power of two");

long long piece_len(long long ckpt) {
    long long P = (long long)std::ceil(std::sqrt(2.0 * (double)ckpt));
    return std::max(1LL, std::min(P, ckpt));
}

bool make_geometry(int S, int C, long long N, long long ckpt, Geometry &g) {
    if (S < 1 || S > kMaxS || C < 1 || N < 1 || ckpt < 1) return false;
    g.N = N;
    g.C = C;
    // shorten the segments while (segments x channels) is below the target
    long long seg = ckpt;
    const long long nt0 = ((N + ckpt - 1) / ckpt) * (long long)C;
    if (nt0 < kTargetThreads) {
        const long long f = (kTargetThreads + nt0 - 1) / nt0;
        seg = std::max(std::min(ckpt, kMinSegment), (ckpt + f - 1) / f);
    }
    g.ckpt = seg;
    g.P = piece_len(seg);
    g.nseg = (N + seg - 1) / seg;
    g.npiece = (std::min(seg, N) + g.P - 1) / g.P;
    g.NT = g.nseg * (long long)C;
    return true;
}

// checkpoints: the state at every piece start, [npiece * 2S][NT]
size_t ckpt_doubles(const Geometry &g, int S) { return (size_t)g.NT * (size_t)(g.npiece * 2 * S); }

// workspace: beta [2S][NT], sig [P*S][NT], gpart [6S][NT], chunk sums [6S][kSumSplit]
size_t work_doubles(const Geometry &g, int S) {
    return (size_t)g.NT * (size_t)(2 * S + g.P * S + 6 * S) + (size_t)(6 * S * kSumSplit);
}

bool check_sos(const double *sos, int S, SosCoef &k) {
    if (!sos || !load_coef(sos, S, k)) {
        set_last_error("sos: NULL, a non-finite coefficient, or a0 == 0");
        return false;
    }
    return true;
}

filark_status launch_status(const char *where) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string(where) + ": " + cudaGetErrorString(e));
        return FILARK_ECUDA;
    }
    return FILARK_OK;
}

template <int S>
void launch_forward(const SosCoef &k, const LocalTables &tb, const Transition &tr, const Geometry &g,
                    const float *x, long long ldx, float *y, long long ldy, double *ckpt, cudaStream_t st) {
    const unsigned nb = (unsigned)((g.NT + kAdjThreads - 1) / kAdjThreads);
    const unsigned nc = (unsigned)((g.C * chain_group<S>() + kChainThreads - 1) / kChainThreads);
    local_block_kernel<S, false><<<nb, kAdjThreads, 0, st>>>(tb, g, x, ldx, ckpt);
    chain_segments_kernel<S><<<nc, kChainThreads, 0, st>>>(tr, g, ckpt, 0);
    fwd_run_kernel<S><<<nb, kAdjThreads, 0, st>>>(k, g, x, ldx, ckpt, y, ldy);
}

template <int S>
void launch_backward(const SosCoef &k, const LocalTables &tb, const Transition &tr, const Geometry &g,
                     const float *x, long long ldx, const float *gy, long long ldg, const double *ckpt, double *work,
                     float *gx, long long ldgx, double *gsos, cudaStream_t st) {
    const unsigned nb = (unsigned)((g.NT + kAdjThreads - 1) / kAdjThreads);
    const unsigned nc = (unsigned)((g.C * chain_group<S>() + kChainThreads - 1) / kChainThreads);
    double *beta = work;
    double *sig = beta + (size_t)g.NT * (2 * S);
    double *gpart = sig + (size_t)g.NT * (size_t)(g.P * S);
    double *chunks = gpart + (size_t)g.NT * (size_t)(6 * S);
    local_block_kernel<S, true><<<nb, kAdjThreads, 0, st>>>(tb, g, gy, ldg, beta);
    chain_segments_kernel<S><<<nc, kChainThreads, 0, st>>>(tr, g, beta, 1);
    adj_run_kernel<S><<<nb, kAdjThreads, 0, st>>>(k, g, x, ldx, gy, ldg, ckpt, beta, sig, gx, ldgx, gpart);
    sum_rows_kernel<<<dim3(6 * S, kSumSplit), kSumThreads, 0, st>>>(gpart, g.NT, g.NT, chunks);
    sum_rows_kernel<<<dim3(6 * S, 1), kSumThreads, 0, st>>>(chunks, kSumSplit, kSumSplit, gsos);
    finish_a0_kernel<<<1, 32, 0, st>>>(k, S, gsos);
}

}  // namespace

extern "C" size_t filark_iir_ckpt_bytes(int n_sections, int n_channels, int64_t n_samples, int64_t ckpt_every) {
    Geometry g;
    if (!make_geometry(n_sections, n_channels, n_samples, ckpt_every, g)) return 0;
    return sizeof(double) * ckpt_doubles(g, n_sections);
}

extern "C" size_t filark_iir_work_bytes(int n_sections, int n_channels, int64_t n_samples, int64_t ckpt_every) {
    Geometry g;
    if (!make_geometry(n_sections, n_channels, n_samples, ckpt_every, g)) return 0;
    return sizeof(double) * work_doubles(g, n_sections);
}

extern "C" filark_status filark_iir_forward_ckpt(const double *sos, int n_sections, int n_channels,
                                                 const float *d_x, int64_t ld_x, int64_t n_samples, float *d_y,
                                                 int64_t ld_y, int64_t ckpt_every, void *d_ckpt, size_t ckpt_size,
                                                 filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_iir_forward_ckpt");
    Geometry g;
    if (!make_geometry(n_sections, n_channels, n_samples, ckpt_every, g)) {
        set_last_error("need 1 <= n_sections <= FILARK_MAX_SECTIONS, n_channels >= 1, n_samples >= 1, ckpt_every >= 1");
        return FILARK_EINVAL;
    }
    SosCoef k;
    if (!check_sos(sos, n_sections, k)) return FILARK_EINVAL;
    if (!d_x || !d_ckpt || ld_x < n_channels || (d_y && ld_y < n_channels)) {
        set_last_error("iir_forward_ckpt: NULL input or checkpoint buffer, or a leading dimension < n_channels");
        return FILARK_EINVAL;
    }
    if (ckpt_size < sizeof(double) * ckpt_doubles(g, n_sections) || ((uintptr_t)d_ckpt & 7)) {
        set_last_error("iir_forward_ckpt: checkpoint buffer smaller than filark_iir_ckpt_bytes or not 8-byte aligned");
        return FILARK_EINVAL;
    }
    Transition tr;
    transition(k, n_sections, false, g.ckpt, tr);
    LocalTables tb;
    local_tables(k, n_sections, false, tb);
    cudaStream_t st = (cudaStream_t)stream;
    double *ck = (double *)d_ckpt;
    switch (n_sections) {
#define FWD_CASE(S_) \
    case S_: launch_forward<S_>(k, tb, tr, g, d_x, ld_x, d_y, ld_y, ck, st); break;
        FWD_CASE(1) FWD_CASE(2) FWD_CASE(3) FWD_CASE(4) FWD_CASE(5) FWD_CASE(6) FWD_CASE(7) FWD_CASE(8)
#undef FWD_CASE
    }
    return launch_status("iir_forward_ckpt");
}

extern "C" filark_status filark_iir_backward(const double *sos, int n_sections, int n_channels, const float *d_x,
                                             int64_t ld_x, int64_t n_samples, const float *d_gy, int64_t ld_gy,
                                             int64_t ckpt_every, const void *d_ckpt, size_t ckpt_size, void *d_work,
                                             size_t work_size, float *d_gx, int64_t ld_gx, double *d_gsos,
                                             filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_iir_backward");
    Geometry g;
    if (!make_geometry(n_sections, n_channels, n_samples, ckpt_every, g)) {
        set_last_error("need 1 <= n_sections <= FILARK_MAX_SECTIONS, n_channels >= 1, n_samples >= 1, ckpt_every >= 1");
        return FILARK_EINVAL;
    }
    SosCoef k;
    if (!check_sos(sos, n_sections, k)) return FILARK_EINVAL;
    if (!d_x || !d_gy || !d_ckpt || !d_work || !d_gsos || ld_x < n_channels || ld_gy < n_channels ||
        (d_gx && ld_gx < n_channels)) {
        set_last_error("iir_backward: NULL buffer or a leading dimension < n_channels");
        return FILARK_EINVAL;
    }
    if (ckpt_size < sizeof(double) * ckpt_doubles(g, n_sections) ||
        work_size < sizeof(double) * work_doubles(g, n_sections) || ((uintptr_t)d_ckpt & 7) ||
        ((uintptr_t)d_work & 7) || ((uintptr_t)d_gsos & 7)) {
        set_last_error("iir_backward: checkpoint or work buffer too small (filark_iir_ckpt_bytes, "
                       "filark_iir_work_bytes) or not 8-byte aligned");
        return FILARK_EINVAL;
    }
    Transition tr;
    transition(k, n_sections, true, g.ckpt, tr);
    LocalTables tb;
    local_tables(k, n_sections, true, tb);
    cudaStream_t st = (cudaStream_t)stream;
    const double *ck = (const double *)d_ckpt;
    double *wk = (double *)d_work;
    switch (n_sections) {
#define BWD_CASE(S_) \
    case S_: launch_backward<S_>(k, tb, tr, g, d_x, ld_x, d_gy, ld_gy, ck, wk, d_gx, ld_gx, d_gsos, st); break;
        BWD_CASE(1) BWD_CASE(2) BWD_CASE(3) BWD_CASE(4) BWD_CASE(5) BWD_CASE(6) BWD_CASE(7) BWD_CASE(8)
#undef BWD_CASE
    }
    return launch_status("iir_backward");
}
