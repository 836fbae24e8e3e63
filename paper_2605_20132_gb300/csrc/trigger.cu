// Triggers and events on the detector ratio (include/filark.h,
// filark_trigger_* and filark_events_*): the monitor stage behind the energy
// detector (Sec. 3.4, threshold detectors behind the monitor interface).
//
// Trigger state per channel, carried across pushes:
//     s(n) = 1 if R(n) >= on,  0 if R(n) < off,  else s(n-1),   s(-1) = 0.
// Every maximal run of s = 1 is a channel trigger [t_on, t_off); it is
// reported by the push in which it ends.  The comparisons are exact: the
// thresholds are rounded up to the nearest float once on the host, and for a
// float R, R >= t holds exactly when R >= (smallest float >= t).
//
// A push is data-parallel over (channel, 32-sample segment):
//   summary  each segment's effect for both incoming states (final state,
//            last rise, whether a run ends inside) -- reads R once;
//   scan     one thread per channel chains the segments (state and the start
//            of the open run), carries the result to the next push, and lists
//            the segments in which a run ends (one atomic per listed segment);
//   emit     one thread per listed segment reads its 32 samples of R again and
//            appends the triggers that end there (one atomic per trigger).
//
// Events are the connected components of the triggers, two triggers being
// joined when their channels are neighbours and their intervals share a
// sample.  The merge buckets the triggers by channel (count, scan, scatter),
// orders each channel's triggers by time, joins overlapping neighbours with a
// lock-free union-find whose roots are the smallest indices, and reduces each
// component to (t_on, t_off, c_min, c_max, n_triggers).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "filark_internal.h"
#include "host_trace.h"

using namespace filark;

namespace {

constexpr int kSeg = 32;          // samples per segment
constexpr int kTrigThreads = 128;
constexpr int kScanThreads = 32;   // one warp per CTA: the scan has only C threads
constexpr int kScanBatch = 16;

// packed segment summary: bits 0/1 final state from 0/1, bits 2/3 a run ends
// inside when entering with 0/1, bits 4-9 / 10-15 last rise + 1 (0 = none)
__device__ __forceinline__ unsigned pack_summary(int f0, int f1, int e0, int e1, int r0, int r1) {
    return (unsigned)f0 | ((unsigned)f1 << 1) | ((unsigned)e0 << 2) | ((unsigned)e1 << 3) |
           ((unsigned)(r0 + 1) << 4) | ((unsigned)(r1 + 1) << 10);
}

__global__ void __launch_bounds__(kTrigThreads) trig_summary_kernel(const float *__restrict__ R, long long ld,
                                                                    int C, int T, float on, float off,
                                                                    unsigned *__restrict__ summ) {
    const int c = blockIdx.x * kTrigThreads + threadIdx.x;
    const int seg = blockIdx.y;
    if (c >= C) return;
    const int a = seg * kSeg, b = min(a + kSeg, T);
    int s0 = 0, s1 = 1, e0 = 0, e1 = 0, r0 = -1, r1 = -1;
#pragma unroll 8
    for (int k = a; k < b; ++k) {
        const float r = R[(long long)k * ld + c];
        const int set = r >= on, reset = r < off;
        const int n0 = set ? 1 : (reset ? 0 : s0);
        const int n1 = set ? 1 : (reset ? 0 : s1);
        r0 = (n0 && !s0) ? k - a : r0;
        r1 = (n1 && !s1) ? k - a : r1;
        e0 |= (!n0 && s0);
        e1 |= (!n1 && s1);
        s0 = n0;
        s1 = n1;
    }
    summ[(size_t)seg * C + c] = pack_summary(s0, s1, e0, e1, r0, r1);
}

// A segment in which a run ends: its channel, index, entry state and the
// start of the run open at its entry.
struct EmitItem {
    long long t_open;
    int c;
    int seg_s;          // segment << 1 | entry state
};

// One thread per channel: chains the segments (the state at each segment
// start), lists the segments in which a run ends, and carries the state.
__global__ void __launch_bounds__(kScanThreads) trig_scan_kernel(const unsigned *__restrict__ summ, int C, int nseg,
                                                                 long long n0, int *__restrict__ st_s,
                                                                 long long *__restrict__ st_t,
                                                                 EmitItem *__restrict__ list,
                                                                 unsigned *__restrict__ list_n) {
    const int c = blockIdx.x * kScanThreads + threadIdx.x;
    if (c >= C) return;
    int s = st_s[c];
    long long t = st_t[c];
    // the summaries do not depend on the chained state: load them kScanBatch
    // at a time, then chain in registers
    for (int g0 = 0; g0 < nseg; g0 += kScanBatch) {
        unsigned m[kScanBatch];
#pragma unroll
        for (int q = 0; q < kScanBatch; ++q) m[q] = g0 + q < nseg ? __ldcs(summ + (size_t)(g0 + q) * C + c) : 0u;
#pragma unroll
        for (int q = 0; q < kScanBatch; ++q) {
            const int g = g0 + q;
            if (g < nseg) {
                if ((m[q] >> (2 + s)) & 1) {
                    const unsigned i = atomicAdd(list_n, 1u);
                    EmitItem it;
                    it.t_open = t;
                    it.c = c;
                    it.seg_s = (g << 1) | s;
                    list[i] = it;
                }
                const int f = (m[q] >> s) & 1;
                const int rise = (int)((m[q] >> (s ? 10 : 4)) & 63) - 1;
                if (f) t = rise >= 0 ? n0 + (long long)g * kSeg + rise : t;
                s = f;
            }
        }
    }
    st_s[c] = s;
    st_t[c] = t;
}

__device__ __forceinline__ void append_record(filark_trigger_record *recs, long long cap,
                                              unsigned long long *count, long long t_on, long long t_off, int c,
                                              int flags) {
    const unsigned long long i = atomicAdd(count, 1ull);
    if ((long long)i < cap) {
        filark_trigger_record r;
        r.t_on = t_on;
        r.t_off = t_off;
        r.channel = c;
        r.flags = flags;
        recs[i] = r;
    }
}

// The listed segments: their samples in flight at once, then the automaton
// from the entry state, appending the triggers that end there.  Grid-stride
// over the list; the first thread also clears the other list counter, which
// the next push uses.
__global__ void __launch_bounds__(kTrigThreads) trig_emit_kernel(const float *__restrict__ R, long long ld, int T,
                                                                 float on, float off, long long n0,
                                                                 const EmitItem *__restrict__ list,
                                                                 unsigned *__restrict__ list_n, int par,
                                                                 filark_trigger_record *__restrict__ recs,
                                                                 long long cap, unsigned long long *count) {
    const unsigned n = list_n[par];
    if (blockIdx.x == 0 && threadIdx.x == 0) list_n[par ^ 1] = 0u;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const EmitItem it = list[i];
        const int c = it.c, seg = it.seg_s >> 1;
        int s = it.seg_s & 1;
        long long t = it.t_open;
        const int a = seg * kSeg, nk = min(kSeg, T - a);
        float rv[kSeg];
#pragma unroll
        for (int k = 0; k < kSeg; ++k) rv[k] = k < nk ? __ldg(R + (long long)(a + k) * ld + c) : 0.f;
#pragma unroll
        for (int k = 0; k < kSeg; ++k) {
            if (k < nk) {
                const float r = rv[k];
                const int nx = r >= on ? 1 : (r < off ? 0 : s);
                if (nx && !s) t = n0 + a + k;
                if (!nx && s) append_record(recs, cap, count, t, n0 + a + k, c, 0);
                s = nx;
            }
        }
    }
}

__global__ void __launch_bounds__(kTrigThreads) trig_flush_kernel(const int *__restrict__ st_s,
                                                                  const long long *__restrict__ st_t, int C,
                                                                  long long n_end,
                                                                  filark_trigger_record *__restrict__ recs,
                                                                  long long cap, unsigned long long *count) {
    const int c = blockIdx.x * kTrigThreads + threadIdx.x;
    if (c >= C || !st_s[c]) return;
    append_record(recs, cap, count, st_t[c], n_end, c, FILARK_TRIGGER_OPEN);
}

// ------------------------------------------------------------ event merge --

struct MergeWork {
    long long *bucket;      // [C + 1] counts, then offsets
    long long *cursor;      // [C]
    long long *ton, *toff;  // [n] triggers bucketed by channel, time-ordered in a bucket
    int *ch, *flg;          // [n]
    long long *parent;      // [n] union-find
    long long *e_ton, *e_toff;  // [n] per-root reductions
    int *e_cmin, *e_cmax, *e_cnt, *e_flg;
    int *bad;               // [1] 1: a channel out of range, 2: union gave up
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

size_t merge_layout(long long n, int C, MergeWork *w, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    const size_t nn = (size_t)(n > 0 ? n : 1);
    MergeWork t;
    t.bucket = (long long *)take(sizeof(long long) * ((size_t)C + 1));
    t.cursor = (long long *)take(sizeof(long long) * (size_t)C);
    t.ton = (long long *)take(sizeof(long long) * nn);
    t.toff = (long long *)take(sizeof(long long) * nn);
    t.ch = (int *)take(sizeof(int) * nn);
    t.flg = (int *)take(sizeof(int) * nn);
    t.parent = (long long *)take(sizeof(long long) * nn);
    t.e_ton = (long long *)take(sizeof(long long) * nn);
    t.e_toff = (long long *)take(sizeof(long long) * nn);
    t.e_cmin = (int *)take(sizeof(int) * nn);
    t.e_cmax = (int *)take(sizeof(int) * nn);
    t.e_cnt = (int *)take(sizeof(int) * nn);
    t.e_flg = (int *)take(sizeof(int) * nn);
    t.bad = (int *)take(sizeof(int));
    if (w) *w = t;
    return off;
}

__global__ void merge_count_kernel(const filark_trigger_record *__restrict__ recs, long long n, int C,
                                   long long *__restrict__ bucket, int *__restrict__ bad) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = recs[i].channel;
    if (c < 0 || c >= C) {
        atomicExch(bad, 1);
        return;
    }
    atomicAdd((unsigned long long *)&bucket[c], 1ull);
}

// exclusive scan of bucket[0..C) into bucket[0..C], one block of 1024 threads
__global__ void __launch_bounds__(1024) merge_scan_kernel(long long *__restrict__ bucket,
                                                          long long *__restrict__ cursor, int C) {
    __shared__ long long part[1024];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < C; base += 1024) {
        const int i = base + threadIdx.x;
        const long long v = i < C ? bucket[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int d = 1; d < 1024; d <<= 1) {
            const long long add = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0;
            __syncthreads();
            part[threadIdx.x] += add;
            __syncthreads();
        }
        const long long excl = carry + part[threadIdx.x] - v;
        if (i < C) {
            bucket[i] = excl;
            cursor[i] = excl;
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) bucket[C] = carry;
}

__global__ void merge_scatter_kernel(const filark_trigger_record *__restrict__ recs, long long n, MergeWork w) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const filark_trigger_record r = recs[i];
    const long long p = (long long)atomicAdd((unsigned long long *)&w.cursor[r.channel], 1ull);
    w.ton[p] = r.t_on;
    w.toff[p] = r.t_off;
    w.ch[p] = r.channel;
    w.flg[p] = r.flags;
}

// one thread per channel: order its triggers by t_on (insertion sort; a
// channel holds few triggers), then initialise the union-find and reductions
__global__ void merge_sort_kernel(MergeWork w, int C) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const long long a = w.bucket[c], b = w.bucket[c + 1];
    for (long long i = a + 1; i < b; ++i) {
        const long long kon = w.ton[i], koff = w.toff[i];
        const int kf = w.flg[i];
        long long j = i - 1;
        while (j >= a && w.ton[j] > kon) {
            w.ton[j + 1] = w.ton[j];
            w.toff[j + 1] = w.toff[j];
            w.flg[j + 1] = w.flg[j];
            --j;
        }
        w.ton[j + 1] = kon;
        w.toff[j + 1] = koff;
        w.flg[j + 1] = kf;
    }
    for (long long i = a; i < b; ++i) {
        w.parent[i] = i;
        w.e_ton[i] = LLONG_MAX;
        w.e_toff[i] = LLONG_MIN;
        w.e_cmin[i] = INT_MAX;
        w.e_cmax[i] = INT_MIN;
        w.e_cnt[i] = 0;
        w.e_flg[i] = 0;
    }
}

// Parents only ever decrease (a root is hooked under a smaller root), so a
// find terminates; reads go to L2 (__ldcg) to see other SMs' hooks.
__device__ __forceinline__ long long uf_find(long long *parent, long long i) {
    long long p = __ldcg(&parent[i]);
    while (p != i) {
        const long long gp = __ldcg(&parent[p]);
        if (gp != p) parent[i] = gp;   // path halving: any ancestor is a valid parent
        i = p;
        p = __ldcg(&parent[i]);
    }
    return i;
}

// Lock-free union; a failed hook means another thread hooked that root first.
// Every failure is matched by a successful hook elsewhere (at most n - 1), so
// the bound (2^22 unless a test lowers it) is never reached by a correct run;
// if it is, *bad is set and the merge reports FILARK_ETIMEOUT.
__device__ void uf_union(long long *parent, long long a, long long b, int *bad, int max_tries) {
    for (int tries = 0; tries < max_tries; ++tries) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return;
        if (a > b) {
            const long long t = a;
            a = b;
            b = t;
        }
        if ((long long)atomicCAS((unsigned long long *)&parent[b], (unsigned long long)b, (unsigned long long)a) == b)
            return;
    }
    atomicExch(bad, 2);
}

// each trigger joins the overlapping triggers of the next channel
__global__ void merge_union_kernel(MergeWork w, long long n, int C, int *bad, int max_tries) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = w.ch[i];
    if (c + 1 >= C) return;
    const long long a = w.ton[i], b = w.toff[i];
    long long lo = w.bucket[c + 1], hi = w.bucket[c + 2];
    // first trigger of channel c+1 that ends after a (intervals of one
    // channel are disjoint and ordered, so t_off is ordered too)
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (w.toff[mid] > a) hi = mid;
        else lo = mid + 1;
    }
    for (long long j = lo; j < w.bucket[c + 2] && w.ton[j] < b; ++j) uf_union(w.parent, i, j, bad, max_tries);
}

__global__ void merge_reduce_kernel(MergeWork w, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long r = uf_find(w.parent, i);
    atomicMin(&w.e_ton[r], w.ton[i]);
    atomicMax(&w.e_toff[r], w.toff[i]);
    atomicMin(&w.e_cmin[r], w.ch[i]);
    atomicMax(&w.e_cmax[r], w.ch[i]);
    atomicAdd(&w.e_cnt[r], 1);
    if (w.flg[i]) atomicOr(&w.e_flg[r], w.flg[i]);
}

__global__ void merge_emit_kernel(MergeWork w, long long n, filark_event *__restrict__ ev, long long cap,
                                  unsigned long long *n_events) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || w.parent[i] != i) return;
    const unsigned long long k = atomicAdd(n_events, 1ull);
    if ((long long)k < cap) {
        filark_event e;
        e.t_on = w.e_ton[i];
        e.t_off = w.e_toff[i];
        e.c_min = w.e_cmin[i];
        e.c_max = w.e_cmax[i];
        e.n_triggers = w.e_cnt[i];
        e.flags = w.e_flg[i];
        ev[k] = e;
    }
}

// smallest float >= v (v finite)
float float_ceil(double v) {
    float f = (float)v;
    if ((double)f < v) f = std::nextafter(f, INFINITY);
    while ((double)f >= v) {
        const float g = std::nextafter(f, -INFINITY);
        if ((double)g < v) break;
        f = g;
    }
    return f;
}




}  // namespace

struct filark_trigger {
    int device = 0;
    int C = 0;
    double on = 0, off = 0;
    float on_f = 0, off_f = 0;
    long long max_chunk = 0, n = 0;
    int nseg_max = 0;
    int *st_s = nullptr;
    long long *st_t = nullptr;
    unsigned *summ = nullptr;       // [2][nseg_max][C]: the summaries of this push (summ + par * C * nseg_max)
    EmitItem *list = nullptr;       // [C * nseg_max] segments in which a run ends
    unsigned *list_n = nullptr;     // [2] list lengths, alternating between pushes
    int par = 0;
    int emit_ctas = 0;
    // overlap mode: the summaries of a push on s_sum, its scan and emit on
    // s_run, so that the summaries of one push run beside the scan and emit
    // of the previous one; the caller's stream only forks (ev_in) and joins
    int overlap = 0;
    bool pending = false;
    cudaStream_t s_sum = nullptr, s_run = nullptr;
    cudaEvent_t ev_in = nullptr, ev_done = nullptr, ev_sum[2] = {nullptr, nullptr}, ev_scan[2] = {nullptr, nullptr};
};

namespace {

void free_trigger(filark_trigger *t) {
    if (!t) return;
    for (cudaEvent_t e : {t->ev_in, t->ev_done, t->ev_sum[0], t->ev_sum[1], t->ev_scan[0], t->ev_scan[1]})
        if (e) cudaEventDestroy(e);
    for (cudaStream_t q : {t->s_sum, t->s_run})
        if (q) cudaStreamDestroy(q);
    for (void *p : {(void *)t->st_s, (void *)t->st_t, (void *)t->summ, (void *)t->list, (void *)t->list_n})
        if (p) cudaFree(p);
    delete t;
}

}  // namespace

extern "C" {

filark_status filark_trigger_create(int n_channels, double on, double off, int64_t max_chunk, int cuda_device,
                                    filark_trigger **out) {
    if (!out) return fail_with(FILARK_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_channels < 1) return fail_with(FILARK_EINVAL, "n_channels must be >= 1");
    if (!std::isfinite(on) || !std::isfinite(off) || off > on)
        return fail_with(FILARK_EINVAL, "thresholds must be finite with off <= on");
    if (std::fabs(on) > 3.0e38 || std::fabs(off) > 3.0e38) return fail_with(FILARK_EINVAL, "thresholds out of float range");
    if (max_chunk < 1 || max_chunk > (int64_t)kSeg * 65535) return fail_with(FILARK_EINVAL, "max_chunk out of range");
    filark_trigger *t = new (std::nothrow) filark_trigger();
    if (!t) return fail_with(FILARK_ENOMEM, "host allocation failed");
    t->device = cuda_device;
    t->C = n_channels;
    t->on = on;
    t->off = off;
    t->on_f = float_ceil(on);
    t->off_f = float_ceil(off);
    t->max_chunk = max_chunk;
    t->nseg_max = (int)((max_chunk + kSeg - 1) / kSeg);
    DeviceGuard dg(cuda_device);
    if (!dg.ok) {
        delete t;
        return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    }
    const size_t C = (size_t)n_channels, G = (size_t)t->nseg_max;
    if (C * G > 0xFFFFFFFFull) {
        delete t;
        return fail_with(FILARK_ENOSYS, "n_channels x ceil(max_chunk / 32) above 2^32 segments");
    }
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cuda_device);
    t->emit_ctas = 2 * std::max(sms, 1);
    if (e == cudaSuccess) e = cudaMalloc(&t->st_s, sizeof(int) * C);
    if (e == cudaSuccess) e = cudaMalloc(&t->st_t, sizeof(long long) * C);
    if (e == cudaSuccess) e = cudaMalloc(&t->summ, 2 * sizeof(unsigned) * C * G);
    if (e == cudaSuccess) e = cudaMalloc(&t->list, sizeof(EmitItem) * C * G);
    if (e == cudaSuccess) e = cudaMalloc(&t->list_n, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(t->list_n, 0, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(t->st_s, 0, sizeof(int) * C);
    if (e == cudaSuccess) e = cudaMemset(t->st_t, 0, sizeof(long long) * C);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_trigger(t);
        return fail_cuda_with(e, "trigger create");
    }
    *out = t;
    return FILARK_OK;
}

filark_status filark_trigger_push(filark_trigger *t, const float *d_ratio, int64_t ld, int64_t n_samples,
                                  filark_trigger_record *d_records, int64_t capacity, unsigned long long *d_count,
                                  filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_trigger_push");
    if (!t) return fail_with(FILARK_EINVAL, "trigger is NULL");
    if (n_samples < 0 || n_samples > t->max_chunk) return fail_with(FILARK_EINVAL, "n_samples must be in [0, max_chunk]");
    if (n_samples == 0) return FILARK_OK;
    if (!d_ratio || ld < t->C) return fail_with(FILARK_EINVAL, "ratio is NULL or ld < n_channels");
    if (!d_count || capacity < 0 || (capacity > 0 && !d_records))
        return fail_with(FILARK_EINVAL, "records/capacity/count arguments");
    DeviceGuard dg(t->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    const int T = (int)n_samples;
    const int nseg = (T + kSeg - 1) / kSeg;
    const dim3 grid2((unsigned)((t->C + kTrigThreads - 1) / kTrigThreads), (unsigned)nseg);
    unsigned *summ = t->summ + (size_t)t->par * (size_t)t->C * (size_t)t->nseg_max;
    cudaError_t e = cudaSuccess;
    cudaStream_t q_sum = s;
    if (t->overlap) {
        // the summaries fork from the caller's stream and wait for the scan
        // that last read this parity's buffer (two pushes ago)
        q_sum = t->s_sum;
        e = cudaEventRecord(t->ev_in, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(q_sum, t->ev_in, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(q_sum, t->ev_scan[t->par], 0);
        if (e != cudaSuccess) return fail_cuda_with(e, "trigger push: fork");
    }
    trig_summary_kernel<<<grid2, kTrigThreads, 0, q_sum>>>(d_ratio, ld, t->C, T, t->on_f, t->off_f, summ);
    if (t->overlap && (e = cudaEventRecord(t->ev_sum[t->par], q_sum)) != cudaSuccess)
        return fail_cuda_with(e, "trigger push: summaries");
    return trigger_push_summarized(t, d_ratio, ld, n_samples, d_records, capacity, d_count, s);
}

}  // extern "C"

namespace filark {

filark_status trigger_fusion_begin(filark_trigger *t, cudaStream_t stream, TriggerFusion &out) {
    if (t->overlap) {
        const cudaError_t e = cudaStreamWaitEvent(stream, t->ev_scan[t->par], 0);
        if (e != cudaSuccess) return fail_cuda_with(e, "trigger fusion: wait");
    }
    out.summ = t->summ + (size_t)t->par * (size_t)t->C * (size_t)t->nseg_max;
    out.on = t->on_f;
    out.off = t->off_f;
    out.C = t->C;
    out.max_chunk = t->max_chunk;
    out.overlap = t->overlap;
    return FILARK_OK;
}

// Scan and emission of a push whose summaries are in the current parity's
// buffer (written on `stream`, or on s_sum with ev_sum recorded, in the
// overlap mode by filark_trigger_push).
filark_status trigger_push_summarized(filark_trigger *t, const float *d_ratio, long long ld, long long n_samples,
                                      filark_trigger_record *d_records, long long capacity,
                                      unsigned long long *d_count, cudaStream_t s, const cudaEvent_t *deps,
                                      int n_deps) {
    const int T = (int)n_samples;
    const int nseg = (T + kSeg - 1) / kSeg;
    const unsigned grid1 = (unsigned)((t->C + kScanThreads - 1) / kScanThreads);
    unsigned *summ = t->summ + (size_t)t->par * (size_t)t->C * (size_t)t->nseg_max;
    cudaError_t e = cudaSuccess;
    cudaStream_t q_run = s;
    if (t->overlap) {
        q_run = t->s_run;
        // after the caller's work (the fused summaries, outputs' zeroing) and,
        // when filark_trigger_push made them, after the summaries on s_sum
        e = cudaEventRecord(t->ev_in, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(q_run, t->ev_in, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(q_run, t->ev_sum[t->par], 0);
        for (int i = 0; i < n_deps && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(q_run, deps[i], 0);
        if (e != cudaSuccess) return fail_cuda_with(e, "trigger push: fork");
    }
    trig_scan_kernel<<<grid1, kScanThreads, 0, q_run>>>(summ, t->C, nseg, t->n, t->st_s, t->st_t, t->list,
                                                        t->list_n + t->par);
    if (t->overlap) {
        e = cudaEventRecord(t->ev_scan[t->par], q_run);
        if (e != cudaSuccess) return fail_cuda_with(e, "trigger push: scan");
        t->pending = true;
    }
    trig_emit_kernel<<<(unsigned)t->emit_ctas, kTrigThreads, 0, q_run>>>(d_ratio, ld, T, t->on_f, t->off_f, t->n,
                                                                         t->list, t->list_n, t->par, d_records,
                                                                         capacity, d_count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda_with(e, "trigger push");
    t->par ^= 1;
    t->n += n_samples;
    return FILARK_OK;
}

}  // namespace filark

extern "C" {

namespace {

// The caller's stream waits for every overlapped push enqueued so far.
filark_status trigger_join(filark_trigger *t, cudaStream_t s) {
    if (!t->pending) return FILARK_OK;
    cudaError_t e = cudaEventRecord(t->ev_done, t->s_run);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, t->ev_done, 0);
    if (e != cudaSuccess) return fail_cuda_with(e, "trigger join");
    t->pending = false;
    return FILARK_OK;
}

}  // namespace

filark_status filark_trigger_join(filark_trigger *t, filark_stream_t stream) {
    if (!t) return fail_with(FILARK_EINVAL, "trigger is NULL");
    DeviceGuard dg(t->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    return trigger_join(t, (cudaStream_t)stream);
}

filark_status filark_trigger_set_overlap(filark_trigger *t, int overlap) {
    if (!t) return fail_with(FILARK_EINVAL, "trigger is NULL");
    if (overlap != 0 && overlap != 1) return fail_with(FILARK_EINVAL, "overlap must be 0 or 1");
    DeviceGuard dg(t->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    cudaError_t e = cudaSuccess;
    if (overlap && !t->s_sum) {
        e = cudaStreamCreateWithFlags(&t->s_sum, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&t->s_run, cudaStreamNonBlocking);
        for (cudaEvent_t *ev : {&t->ev_in, &t->ev_done, &t->ev_sum[0], &t->ev_sum[1], &t->ev_scan[0], &t->ev_scan[1]})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail_cuda_with(e, "trigger overlap: streams");
    }
    // work already enqueued in the other mode finishes first
    if (t->s_run) {
        e = cudaStreamSynchronize(t->s_run);
        if (e == cudaSuccess) e = cudaStreamSynchronize(t->s_sum);
        if (e != cudaSuccess) return fail_cuda_with(e, "trigger overlap: synchronize");
    }
    t->pending = false;
    t->overlap = overlap;
    return FILARK_OK;
}

filark_status filark_trigger_flush(filark_trigger *t, filark_trigger_record *d_records, int64_t capacity,
                                   unsigned long long *d_count, filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_trigger_flush");
    if (!t) return fail_with(FILARK_EINVAL, "trigger is NULL");
    if (!d_count || capacity < 0 || (capacity > 0 && !d_records))
        return fail_with(FILARK_EINVAL, "records/capacity/count arguments");
    DeviceGuard dg(t->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    const filark_status js = trigger_join(t, (cudaStream_t)stream);
    if (js != FILARK_OK) return js;
    trig_flush_kernel<<<(unsigned)((t->C + kTrigThreads - 1) / kTrigThreads), kTrigThreads, 0,
                        (cudaStream_t)stream>>>(t->st_s, t->st_t, t->C, t->n, d_records, capacity, d_count);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FILARK_OK : fail_cuda_with(e, "trigger flush");
}

filark_status filark_trigger_reset(filark_trigger *t, filark_stream_t stream) {
    if (!t) return fail_with(FILARK_EINVAL, "trigger is NULL");
    DeviceGuard dg(t->device);
    if (!dg.ok) return fail_with(FILARK_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    const filark_status js = trigger_join(t, s);
    if (js != FILARK_OK) return js;
    cudaError_t e = cudaMemsetAsync(t->st_s, 0, sizeof(int) * (size_t)t->C, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->st_t, 0, sizeof(long long) * (size_t)t->C, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->list_n, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return fail_cuda_with(e, "trigger reset");
    t->n = 0;
    return FILARK_OK;
}

filark_status filark_trigger_destroy(filark_trigger *t) {
    if (!t) return FILARK_OK;
    DeviceGuard dg(t->device);
    cudaDeviceSynchronize();
    free_trigger(t);
    return FILARK_OK;
}

size_t filark_events_work_bytes(int64_t n_triggers, int n_channels) {
    if (n_triggers < 0 || n_channels < 1) return 0;
    return merge_layout(n_triggers, n_channels, nullptr, nullptr);
}

filark_status filark_events_merge(const filark_trigger_record *d_triggers, int64_t n_triggers, int n_channels,
                                  filark_event *d_events, int64_t capacity, unsigned long long *d_n_events,
                                  void *d_work, size_t work_bytes, filark_stream_t stream) {
    filark::NvtxRange nvtx_range("filark_events_merge");
    if (n_triggers < 0 || n_channels < 1) return fail_with(FILARK_EINVAL, "n_triggers < 0 or n_channels < 1");
    if (!d_n_events || capacity < 0 || (capacity > 0 && !d_events))
        return fail_with(FILARK_EINVAL, "events/capacity/count arguments");
    if (n_triggers == 0) return FILARK_OK;
    if (!d_triggers || !d_work || work_bytes < filark_events_work_bytes(n_triggers, n_channels) ||
        ((uintptr_t)d_work & 255))
        return fail_with(FILARK_EINVAL, "triggers NULL, or work buffer too small / not 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    MergeWork w;
    merge_layout(n_triggers, n_channels, &w, (char *)d_work);
    int *bad = w.bad;
    cudaError_t e = cudaMemsetAsync(w.bucket, 0, sizeof(long long) * ((size_t)n_channels + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e != cudaSuccess) return fail_cuda_with(e, "events merge: clear");
    const unsigned gn = (unsigned)((n_triggers + 255) / 256);
    merge_count_kernel<<<gn, 256, 0, s>>>(d_triggers, n_triggers, n_channels, w.bucket, bad);
    int bad_h = 0;
    e = cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda_with(e, "events merge: check");
    if (bad_h) return fail_with(FILARK_EINVAL, "a trigger's channel is outside [0, n_channels)");
    merge_scan_kernel<<<1, 1024, 0, s>>>(w.bucket, w.cursor, n_channels);
    merge_scatter_kernel<<<gn, 256, 0, s>>>(d_triggers, n_triggers, w);
    merge_sort_kernel<<<(unsigned)((n_channels + 127) / 128), 128, 0, s>>>(w, n_channels);
    // FILARK_TEST_UNION_TRIES lowers the retry bound so that a test can see
    // the bounded loop give up and the merge report it (never set otherwise)
    int max_tries = 1 << 22;
    if (const char *ev = std::getenv("FILARK_TEST_UNION_TRIES")) max_tries = std::max(0, std::atoi(ev));
    merge_union_kernel<<<gn, 256, 0, s>>>(w, n_triggers, n_channels, bad, max_tries);
    merge_reduce_kernel<<<gn, 256, 0, s>>>(w, n_triggers);
    merge_emit_kernel<<<gn, 256, 0, s>>>(w, n_triggers, d_events, capacity, d_n_events);
    e = cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda_with(e, "events merge");
    if (bad_h) return fail_with(FILARK_ETIMEOUT, "events merge: union-find gave up");
    return FILARK_OK;
}

}  // extern "C"
