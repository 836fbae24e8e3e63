// Host planner of the chunked DAS filter chain.
//
// The IIR stage of the chain is a cascade of S second-order sections in
// transposed direct form II (Table 1 of the paper: realtime SOS filter).  The
// GPU does not run that recurrence sample by sample.  It runs the equivalent
// block state-space form of the whole cascade:
//
//   state s (2S values: z1, z2 of every section), s[n+1] = A s[n] + B x[n],
//   y[n] = C s[n] + D x[n].  For a block of L samples starting in state s_j:
//       y_j[k]  = sum_{i<=k} h[k-i] x_j[i] + (C A^k) s_j          (k < L)
//       s_{j+1} = A^L s_j + sum_i A^(L-1-i) B x_j[i]
//   with h[0] = D, h[m] = C A^(m-1) B.
//
// so that every block can be processed in parallel and only the short carry
// recurrence s_{j+1} = A^L s_j + e_j is sequential.  The carry is diagonalised:
// A = W M W^-1 with M block-diagonal (one 2x2 block per conjugate pole pair, or
// per pair of real poles), so the carry costs 4 multiply-adds per slot and
// block.  All tables are derived in long double and rounded to FP32 once; the
// carry is kept in FP64 between thread blocks and chunks.
//
// Rounding the recurrence coefficients themselves to FP32 moves poles that lie
// close to z = 1 (the 0.5 Hz sections of a 1.5 kHz bandpass sit 4e-4 from the
// unit circle) far enough to change the filter by ~1e-3; the block tables do not
// have that sensitivity, which is why this form is used.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstring>
#include <limits>

#include "filark_internal.h"

namespace filark {

using ld = long double;
using cld = std::complex<long double>;

namespace {

// Normalised section: y = b0 u + z1; z1' = b1 u - a1 y + z2; z2' = b2 u - a2 y.
struct Section {
    ld b0, b1, b2, a1, a2;
};

// Poles of z^2 + a1 z + a2 (numerically stable quadratic formula).
void section_poles(const Section &s, cld &p1, cld &p2) {
    ld disc = s.a1 * s.a1 - 4 * s.a2;
    if (disc < 0) {
        ld re = -s.a1 / 2, im = std::sqrt(-disc) / 2;
        p1 = cld(re, im);
        p2 = cld(re, -im);
    } else {
        ld sq = std::sqrt(disc);
        ld q = -(s.a1 + (s.a1 >= 0 ? sq : -sq)) / 2;
        if (q == 0) {
            p1 = p2 = cld(0, 0);
        } else {
            p1 = cld(q, 0);
            p2 = cld(s.a2 / q, 0);
        }
    }
}

// One TDF-II step of the whole cascade on a long double state (used to read
// off A, B, C, D column by column).
ld cascade_step(const std::vector<Section> &secs, std::vector<ld> &z, ld u) {
    for (size_t s = 0; s < secs.size(); ++s) {
        const Section &k = secs[s];
        ld y = k.b0 * u + z[2 * s];
        ld z1 = k.b1 * u - k.a1 * y + z[2 * s + 1];
        ld z2 = k.b2 * u - k.a2 * y;
        z[2 * s] = z1;
        z[2 * s + 1] = z2;
        u = y;
    }
    return u;
}

bool invert(std::vector<ld> a, int n, std::vector<ld> &inv) {
    inv.assign((size_t)n * n, 0);
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(a[(size_t)r * n + col]) > std::fabs(a[(size_t)piv * n + col])) piv = r;
        if (a[(size_t)piv * n + col] == 0) return false;
        if (piv != col) {
            for (int c = 0; c < n; ++c) {
                std::swap(a[(size_t)piv * n + c], a[(size_t)col * n + c]);
                std::swap(inv[(size_t)piv * n + c], inv[(size_t)col * n + c]);
            }
        }
        ld d = a[(size_t)col * n + col];
        for (int c = 0; c < n; ++c) {
            a[(size_t)col * n + c] /= d;
            inv[(size_t)col * n + c] /= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            ld f = a[(size_t)r * n + col];
            if (f == 0) continue;
            for (int c = 0; c < n; ++c) {
                a[(size_t)r * n + c] -= f * a[(size_t)col * n + c];
                inv[(size_t)r * n + c] -= f * inv[(size_t)col * n + c];
            }
        }
    }
    return true;
}

ld frob(const std::vector<ld> &a) {
    ld s = 0;
    for (ld v : a) s += v * v;
    return std::sqrt(s);
}

// Emulates, on one channel, the FP32/FP64 arithmetic the kernel performs, and
// returns the normwise error against a long double TDF-II run of the same
// input.  Used to verify the FP32 modal tables before a chain is accepted.
// fewest_blocks: every launch uses the fewest blocks per CTA a caller may set
// (more CTAs, shorter FP32 chains) instead of kNB.
double probe_modal(const Plan &pl, const std::vector<Section> &secs, bool fewest_blocks) {
    const int NS = pl.NS, R2 = 2 * NS;
    // deterministic probe: uniform noise with an impulse at the start
    const int launches[] = {2048, 1500, 1, 700, 2048, 33, 2048};
    int N = 0;
    for (int t : launches) N += t;
    std::vector<float> x((size_t)N);
    uint64_t st = 0x9E3779B97F4A7C15ull;
    for (int n = 0; n < N; ++n) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        x[(size_t)n] = (float)((double)(st >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
    }
    x[0] = 8.0f;
    // reference
    std::vector<ld> z(2 * secs.size(), 0);
    std::vector<double> yref((size_t)N);
    for (int n = 0; n < N; ++n) yref[(size_t)n] = (double)cascade_step(secs, z, (ld)x[(size_t)n]);
    // emulation
    std::vector<double> yemu((size_t)N);
    std::vector<double> state((size_t)R2, 0.0);
    double Mr[kMaxSlots][4];
    const Tables32 &tb = pl.tab;
    int base = 0;
    for (int T : launches) {
        const int nblk = (T + kL - 1) / kL, Lr = T - (nblk - 1) * kL;
        pl.slot_power(Lr, Mr);
        const int nbc = fewest_blocks ? std::max(1, (nblk + kMaxCluster - 1) / kMaxCluster) : kNB;
        const int R = (nblk + nbc - 1) / nbc;
        std::vector<float> e((size_t)nblk * R2), er((size_t)R2, 0.f);
        std::vector<float> yl((size_t)nblk * kL);
        for (int j = 0; j < nblk; ++j) {
            float xb[kL];
            for (int i = 0; i < kL; ++i) {
                int row = j * kL + i;
                xb[i] = row < T ? x[(size_t)(base + row)] : 0.f;
            }
            for (int k = 0; k < kL; ++k) {
                float acc = 0.f;
                for (int i = 0; i <= k; ++i) acc = std::fmaf(tb.h[k - i], xb[i], acc);
                yl[(size_t)j * kL + k] = acc;
            }
            for (int r = 0; r < R2; ++r) {
                float acc = 0.f;
                for (int i = 0; i < kL; ++i) acc = std::fmaf(tb.K[i][r], xb[i], acc);
                e[(size_t)j * R2 + r] = acc;
            }
            if (j == nblk - 1 && Lr < kL) {
                for (int r = 0; r < R2; ++r) {
                    float acc = 0.f;
                    for (int i = kL - Lr; i < kL; ++i) acc = std::fmaf(tb.K[i][r], xb[i - (kL - Lr)], acc);
                    er[(size_t)r] = acc;
                }
            }
        }
        // carries: FP32 aggregate per CTA (the last CTA's ragged block uses
        // M^Lr and the right-aligned end state), FP64 across CTAs and launches
        const int nb_last = nblk - (R - 1) * nbc;
        double PhiLast[kMaxSlots][4];
        pl.slot_power((nb_last - 1) * kL + Lr, PhiLast);
        std::vector<float> agg((size_t)R * R2, 0.f);
        for (int rr = 0; rr < R; ++rr) {
            int j0 = rr * nbc, nb = std::min(nbc, nblk - j0);
            for (int s = 0; s < NS; ++s) {
                float a0 = 0.f, a1 = 0.f;
                for (int jj = 0; jj < nb; ++jj) {
                    const bool rag = (rr == R - 1) && (jj == nb - 1) && Lr < kL;
                    float M[4];
                    for (int q = 0; q < 4; ++q) M[q] = rag ? (float)Mr[s][q] : tb.M[s][q];
                    float e0 = rag ? er[(size_t)2 * s] : e[(size_t)(j0 + jj) * R2 + 2 * s];
                    float e1 = rag ? er[(size_t)2 * s + 1] : e[(size_t)(j0 + jj) * R2 + 2 * s + 1];
                    float t0 = std::fmaf(M[0], a0, std::fmaf(M[1], a1, e0));
                    float t1 = std::fmaf(M[2], a0, std::fmaf(M[3], a1, e1));
                    a0 = t0;
                    a1 = t1;
                }
                agg[(size_t)rr * R2 + 2 * s] = a0;
                agg[(size_t)rr * R2 + 2 * s + 1] = a1;
            }
        }
        std::vector<float> mstart((size_t)nblk * R2);
        std::vector<double> newstate((size_t)R2);
        const double (*PP)[4] = pl.power_cached_cta(nbc, R - 1);
        for (int rr = 0; rr < R; ++rr) {
            int j0 = rr * nbc, nb = std::min(nbc, nblk - j0);
            const double (*Pr)[4] = pl.power_cached_cta(nbc, rr);
            for (int s = 0; s < NS; ++s) {
                // as the kernel: earlier CTAs' aggregates through their own FP32
                // powers, the carried state's leading float through Phi^rr
                float g0 = 0.f, g1 = 0.f;
                for (int q = 0; q < rr; ++q) {
                    const double (*Pq)[4] = pl.power_cached_cta(nbc, rr - 1 - q);
                    const float a0 = agg[(size_t)q * R2 + 2 * s], a1 = agg[(size_t)q * R2 + 2 * s + 1];
                    g0 = std::fmaf((float)Pq[s][0], a0, std::fmaf((float)Pq[s][1], a1, g0));
                    g1 = std::fmaf((float)Pq[s][2], a0, std::fmaf((float)Pq[s][3], a1, g1));
                }
                const double c0 = state[(size_t)2 * s], c1 = state[(size_t)2 * s + 1];
                const float c0h = (float)c0, c1h = (float)c1;
                float f0 = std::fmaf((float)Pr[s][0], c0h, std::fmaf((float)Pr[s][1], c1h, g0));
                float f1 = std::fmaf((float)Pr[s][2], c0h, std::fmaf((float)Pr[s][3], c1h, g1));
                if (rr == R - 1) {
                    // end state PhiTot c + PhiLast g + own aggregate (double-float
                    // in the kernel, double here)
                    const double *a = PhiLast[s], *b = PP[s];
                    const double T0 = a[0] * b[0] + a[1] * b[2], T1 = a[0] * b[1] + a[1] * b[3];
                    const double T2 = a[2] * b[0] + a[3] * b[2], T3 = a[2] * b[1] + a[3] * b[3];
                    const double o0 = agg[(size_t)rr * R2 + 2 * s], o1 = agg[(size_t)rr * R2 + 2 * s + 1];
                    newstate[(size_t)2 * s] = T0 * c0 + T1 * c1 + (a[0] * g0 + a[1] * g1) + o0;
                    newstate[(size_t)2 * s + 1] = T2 * c0 + T3 * c1 + (a[2] * g0 + a[3] * g1) + o1;
                }
                const float *M = tb.M[s];
                for (int jj = 0; jj < nb; ++jj) {
                    int j = j0 + jj;
                    float e0 = e[(size_t)j * R2 + 2 * s], e1 = e[(size_t)j * R2 + 2 * s + 1];
                    mstart[(size_t)j * R2 + 2 * s] = f0;
                    mstart[(size_t)j * R2 + 2 * s + 1] = f1;
                    float t0 = std::fmaf(M[0], f0, std::fmaf(M[1], f1, e0));
                    float t1 = std::fmaf(M[2], f0, std::fmaf(M[3], f1, e1));
                    f0 = t0;
                    f1 = t1;
                }
            }
        }
        state = newstate;
        for (int j = 0; j < nblk; ++j) {
            for (int k = 0; k < kL; ++k) {
                int row = j * kL + k;
                if (row >= T) break;
                float acc = yl[(size_t)j * kL + k];
                for (int r = 0; r < R2; ++r) acc = std::fmaf(tb.G[k][r], mstart[(size_t)j * R2 + r], acc);
                yemu[(size_t)(base + row)] = acc;
            }
        }
        base += T;
    }
    double num = 0, den = 0;
    for (int n = 0; n < N; ++n) {
        num = std::max(num, std::fabs(yemu[(size_t)n] - yref[(size_t)n]));
        den = std::max(den, std::fabs(yref[(size_t)n]));
    }
    if (!(num == num)) return std::numeric_limits<double>::infinity();
    return den > 0 ? num / den : num;
}

// Same check for the dense carry: FP32 tables in the canonical basis, an FP64
// carry at every block, the block start state rounded to FP32 for the fix-up.
double probe_dense(const Plan &pl, const std::vector<Section> &secs, const std::vector<ld> &Acan) {
    const int n = 2 * pl.S;
    const int N = 6144;
    std::vector<float> x((size_t)N);
    uint64_t st = 0x2545F4914F6CDD1Dull;
    for (int i = 0; i < N; ++i) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        x[(size_t)i] = (float)((double)(st >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
    }
    x[0] = 8.0f;
    std::vector<ld> z(2 * secs.size(), 0);
    std::vector<double> yref((size_t)N), yemu((size_t)N);
    for (int i = 0; i < N; ++i) yref[(size_t)i] = (double)cascade_step(secs, z, (ld)x[(size_t)i]);
    // A^L in FP64
    std::vector<double> AL((size_t)n * n);
    {
        std::vector<ld> P((size_t)n * n, 0), Q;
        for (int i = 0; i < n; ++i) P[(size_t)i * n + i] = 1;
        for (int k = 0; k < kL; ++k) {
            Q.assign((size_t)n * n, 0);
            for (int r = 0; r < n; ++r)
                for (int c = 0; c < n; ++c)
                    for (int q = 0; q < n; ++q) Q[(size_t)r * n + c] += Acan[(size_t)r * n + q] * P[(size_t)q * n + c];
            P = Q;
        }
        for (size_t i = 0; i < AL.size(); ++i) AL[i] = (double)P[i];
    }
    const Tables32 &tb = pl.tab;
    std::vector<double> m((size_t)n, 0.0);
    for (int j = 0; j * kL < N; ++j) {
        float mf[kDenseDim];
        for (int r = 0; r < n; ++r) mf[r] = (float)m[(size_t)r];
        float e[kDenseDim];
        for (int r = 0; r < n; ++r) e[r] = 0.f;
        for (int k = 0; k < kL; ++k) {
            float acc = 0.f;
            for (int i = 0; i <= k; ++i) acc = std::fmaf(tb.h[k - i], x[(size_t)(j * kL + i)], acc);
            for (int r = 0; r < n; ++r) acc = std::fmaf(tb.G[k][r], mf[r], acc);
            yemu[(size_t)(j * kL + k)] = acc;
        }
        for (int r = 0; r < n; ++r)
            for (int i = 0; i < kL; ++i) e[r] = std::fmaf(tb.K[i][r], x[(size_t)(j * kL + i)], e[r]);
        std::vector<double> nm((size_t)n, 0.0);
        for (int r = 0; r < n; ++r) {
            double acc = (double)e[r];
            for (int q = 0; q < n; ++q) acc = std::fma(AL[(size_t)r * n + q], m[(size_t)q], acc);
            nm[(size_t)r] = acc;
        }
        m = nm;
    }
    double num = 0, den = 0;
    for (int i = 0; i < N; ++i) {
        num = std::max(num, std::fabs(yemu[(size_t)i] - yref[(size_t)i]));
        den = std::max(den, std::fabs(yref[(size_t)i]));
    }
    if (!(num == num)) return std::numeric_limits<double>::infinity();
    return den > 0 ? num / den : num;
}

// Dense matrices for the kernel: A^1..A^L and Phi^0..Phi^(kMaxCluster-1),
// Phi = A^(L*kNB), each padded to kDenseDim x kDenseDim.
std::vector<double> dense_matrices(const std::vector<ld> &A, int n) {
    const int D = kDenseDim;
    std::vector<double> out((size_t)kDenseMats * D * D, 0.0);
    auto mul = [&](const std::vector<ld> &X, const std::vector<ld> &Y) {
        std::vector<ld> Z((size_t)n * n, 0);
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < n; ++c) {
                ld acc = 0;
                for (int q = 0; q < n; ++q) acc += X[(size_t)r * n + q] * Y[(size_t)q * n + c];
                Z[(size_t)r * n + c] = acc;
            }
        return Z;
    };
    auto put = [&](int slot, const std::vector<ld> &M) {
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < n; ++c) out[((size_t)slot * D + r) * D + c] = (double)M[(size_t)r * n + c];
    };
    std::vector<ld> P = A;
    for (int k = 1; k <= kL; ++k) {
        put(k - 1, P);
        if (k < kL) P = mul(P, A);
    }
    std::vector<ld> Phi = P;                       // A^L
    for (int k = 1; k < kNB; ++k) Phi = mul(Phi, P);  // A^(L*kNB)
    std::vector<ld> Q((size_t)n * n, 0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1;
    for (int r = 0; r < kMaxCluster; ++r) {
        put(kL + r, Q);
        Q = mul(Q, Phi);
    }
    return out;
}

// The kernel's layout of the dense matrices.  A column's state (n = 2NS rows)
// lives in 8 lanes of a warp, lane w < NS holding rows w and n-1-w; at step q
// of a matrix-vector product every lane takes the entries (w, q) and
// (n-1-w, q) as one float4 {hi, lo of row w; hi, lo of row n-1-w}, a
// double-float split of the FP64 entry.  Output [kDenseMats][kDenseDim][8]
// float4.  The powers of the cascade's transition matrix are block lower
// triangular (section k depends only on sections <= k), so row w needs the
// columns q < NS only and the kernel reads no other entry of it; false if an
// entry it would skip is not zero.
bool dense_lane_layout(const std::vector<double> &mats, int NS, std::vector<float> &out) {
    const int D = kDenseDim, n = 2 * NS;
    out.assign((size_t)kDenseMats * D * 8 * 4, 0.f);
    auto split = [](double v, float *dst) {
        const float hi = (float)v;
        dst[0] = hi;
        dst[1] = (float)(v - (double)hi);
    };
    for (int m = 0; m < kDenseMats; ++m) {
        const double *M = mats.data() + (size_t)m * D * D;
        for (int w = 0; w < NS; ++w)
            for (int q = NS; q < n; ++q)
                if (M[(size_t)w * D + q] != 0.0) return false;
        for (int q = 0; q < n; ++q)
            for (int w = 0; w < NS; ++w) {
                float *f = out.data() + (((size_t)m * D + q) * 8 + w) * 4;
                if (q < NS) split(M[(size_t)w * D + q], f);
                split(M[(size_t)(n - 1 - w) * D + q], f + 2);
            }
    }
    return true;
}

}  // namespace

void Plan::slot_power(int n, double out[kMaxSlots][4]) const {
    for (int s = 0; s < kMaxSlots; ++s) {
        out[s][0] = out[s][1] = out[s][2] = out[s][3] = 0.0;
        if (s >= S) continue;
        if (slot_kind[s] == 0) {
            cld lam(slot_a[s], slot_b[s]), p(1, 0);
            // repeated squaring in long double
            cld base = lam;
            for (int e = n; e > 0; e >>= 1) {
                if (e & 1) p *= base;
                base *= base;
            }
            out[s][0] = (double)p.real();
            out[s][1] = (double)p.imag();
            out[s][2] = (double)(-p.imag());
            out[s][3] = (double)p.real();
        } else {
            ld pa = 1, pb = 1, ba = slot_a[s], bb = slot_b[s];
            for (int e = n; e > 0; e >>= 1) {
                if (e & 1) {
                    pa *= ba;
                    pb *= bb;
                }
                ba *= ba;
                bb *= bb;
            }
            out[s][0] = (double)pa;
            out[s][3] = (double)pb;
        }
    }
}

const double (*Plan::power_cached(int n) const)[4] {
    if (pow_cache.empty()) {
        pow_cache.assign((size_t)(kTileRows + 1) * kMaxSlots * 4, 0.0);
        pow_have.assign((size_t)(kTileRows + 1), 0);
    }
    double (*slot)[4] = reinterpret_cast<double (*)[4]>(&pow_cache[(size_t)n * kMaxSlots * 4]);
    if (!pow_have[(size_t)n]) {
        slot_power(n, slot);
        pow_have[(size_t)n] = 1;
    }
    return slot;
}

const double (*Plan::power_cached_cta(int nbc, int r) const)[4] {
    if (cta_cache.empty()) {
        cta_cache.assign((size_t)(kNB + 1) * kMaxCluster * kMaxSlots * 4, 0.0);
        cta_have.assign((size_t)(kNB + 1), 0);
    }
    double *base = &cta_cache[(size_t)nbc * kMaxCluster * kMaxSlots * 4];
    if (!cta_have[(size_t)nbc]) {
        for (int q = 0; q < kMaxCluster; ++q)
            slot_power(kL * nbc * q, reinterpret_cast<double (*)[4]>(base + (size_t)q * kMaxSlots * 4));
        cta_have[(size_t)nbc] = 1;
    }
    return reinterpret_cast<const double (*)[4]>(base + (size_t)r * kMaxSlots * 4);
}

filark_status make_plan(const double *sos, int S, int precision, Plan *pl, std::string *err) {
    *pl = Plan();
    pl->S = S;
    if (S == 0) {
        pl->NS = 0;
        pl->mode = FILARK_PREC_MODAL32;
        return FILARK_OK;
    }
    pl->NS = S <= 2 ? 2 : (S <= 4 ? 4 : 8);
    std::vector<Section> secs((size_t)S);
    for (int s = 0; s < S; ++s) {
        const double *r = sos + 6 * s;
        for (int i = 0; i < 6; ++i) {
            if (!std::isfinite(r[i])) {
                *err = "sos: non-finite coefficient in section " + std::to_string(s);
                return FILARK_EINVAL;
            }
        }
        if (r[3] == 0.0) {
            *err = "sos: a0 == 0 in section " + std::to_string(s);
            return FILARK_EINVAL;
        }
        ld a0 = r[3];
        secs[(size_t)s] = Section{(ld)r[0] / a0, (ld)r[1] / a0, (ld)r[2] / a0, (ld)r[4] / a0, (ld)r[5] / a0};
        cld p1, p2;
        section_poles(secs[(size_t)s], p1, p2);
        if (!(std::abs(p1) < 1) || !(std::abs(p2) < 1)) {
            *err = "sos: section " + std::to_string(s) + " has a pole on or outside the unit circle";
            return FILARK_EUNSTABLE;
        }
    }
    const int n = 2 * S;
    // canonical state space, read off the TDF-II recurrence
    std::vector<ld> A((size_t)n * n), B((size_t)n), Cr((size_t)n);
    ld D;
    for (int i = 0; i < n; ++i) {
        std::vector<ld> z((size_t)n, 0);
        z[(size_t)i] = 1;
        Cr[(size_t)i] = cascade_step(secs, z, 0);
        for (int r = 0; r < n; ++r) A[(size_t)r * n + i] = z[(size_t)r];
    }
    {
        std::vector<ld> z((size_t)n, 0);
        D = cascade_step(secs, z, 1);
        for (int r = 0; r < n; ++r) B[(size_t)r] = z[(size_t)r];
    }
    // modal basis: eigenvectors by forward substitution over the block lower
    // triangular A (section q depends only on sections <= q)
    std::vector<ld> W((size_t)n * n, 0);
    bool modal_ok = true;
    auto eigvec = [&](int s, cld lam, std::vector<cld> &v) -> bool {
        v.assign((size_t)n, cld(0, 0));
        v[(size_t)2 * s] = 1;
        v[(size_t)2 * s + 1] = lam + secs[(size_t)s].a1;
        for (int q = s + 1; q < S; ++q) {
            cld rhs0 = 0, rhs1 = 0;
            for (int t = 0; t < 2 * q; ++t) {
                rhs0 -= A[(size_t)(2 * q) * n + t] * v[(size_t)t];
                rhs1 -= A[(size_t)(2 * q + 1) * n + t] * v[(size_t)t];
            }
            cld m00 = A[(size_t)(2 * q) * n + 2 * q] - lam, m01 = A[(size_t)(2 * q) * n + 2 * q + 1];
            cld m10 = A[(size_t)(2 * q + 1) * n + 2 * q], m11 = A[(size_t)(2 * q + 1) * n + 2 * q + 1] - lam;
            cld det = m00 * m11 - m01 * m10;
            ld scale = std::abs(m00) * std::abs(m11) + std::abs(m01) * std::abs(m10) + 1e-300L;
            if (std::abs(det) < 1e-14L * scale) return false;
            v[(size_t)2 * q] = (rhs0 * m11 - m01 * rhs1) / det;
            v[(size_t)2 * q + 1] = (m00 * rhs1 - m10 * rhs0) / det;
        }
        return true;
    };
    for (int s = 0; s < S && modal_ok; ++s) {
        cld p1, p2;
        section_poles(secs[(size_t)s], p1, p2);
        std::vector<cld> v1, v2;
        if (p1.imag() != 0) {
            cld lam = p1.imag() > 0 ? p1 : p2;
            if (!eigvec(s, lam, v1)) { modal_ok = false; break; }
            for (int r = 0; r < n; ++r) {
                W[(size_t)r * n + 2 * s] = v1[(size_t)r].real();
                W[(size_t)r * n + 2 * s + 1] = v1[(size_t)r].imag();
            }
            pl->slot_kind[s] = 0;
            pl->slot_a[s] = lam.real();
            pl->slot_b[s] = lam.imag();
        } else {
            if (p1 == p2) { modal_ok = false; break; }   // repeated real pole: defective
            if (!eigvec(s, p1, v1) || !eigvec(s, p2, v2)) { modal_ok = false; break; }
            for (int r = 0; r < n; ++r) {
                W[(size_t)r * n + 2 * s] = v1[(size_t)r].real();
                W[(size_t)r * n + 2 * s + 1] = v2[(size_t)r].real();
            }
            pl->slot_kind[s] = 1;
            pl->slot_a[s] = p1.real();
            pl->slot_b[s] = p2.real();
        }
    }
    std::vector<ld> Winv;
    if (modal_ok && !invert(W, n, Winv)) modal_ok = false;
    if (precision == FILARK_PREC_MODAL32 && !modal_ok) {
        *err = "the IIR cascade has repeated poles (no modal basis)";
        return FILARK_ENOSYS;
    }
    // full tables in the canonical basis
    std::vector<ld> h((size_t)kL), Kf((size_t)n * kL), Gf((size_t)kL * n);
    {
        h[0] = D;
        std::vector<std::vector<ld>> pw((size_t)kL);   // pw[m] = A^m B
        pw[0] = B;
        for (int m = 1; m < kL; ++m) {
            pw[(size_t)m].assign((size_t)n, 0);
            for (int r = 0; r < n; ++r) {
                ld acc = 0;
                for (int c = 0; c < n; ++c) acc += A[(size_t)r * n + c] * pw[(size_t)m - 1][(size_t)c];
                pw[(size_t)m][(size_t)r] = acc;
            }
        }
        for (int m = 1; m < kL; ++m) {
            ld acc = 0;
            for (int r = 0; r < n; ++r) acc += Cr[(size_t)r] * pw[(size_t)m - 1][(size_t)r];
            h[(size_t)m] = acc;
        }
        for (int i = 0; i < kL; ++i)
            for (int r = 0; r < n; ++r) Kf[(size_t)r * kL + i] = pw[(size_t)(kL - 1 - i)][(size_t)r];
        std::vector<ld> w(Cr);         // C A^k
        for (int k = 0; k < kL; ++k) {
            for (int c = 0; c < n; ++c) Gf[(size_t)k * n + c] = w[(size_t)c];
            std::vector<ld> nw((size_t)n, 0);
            for (int c = 0; c < n; ++c)
                for (int r = 0; r < n; ++r) nw[(size_t)c] += w[(size_t)r] * A[(size_t)r * n + c];
            w = nw;
        }
    }
    Tables32 &tb = pl->tab;
    auto fill_tables = [&](const std::vector<ld> &Km, const std::vector<ld> &Gm) {
        std::memset(&tb, 0, sizeof(tb));
        for (int k = 0; k < kL; ++k) tb.h[k] = (float)h[(size_t)k];
        for (int i = 0; i < kL; ++i)
            for (int r = 0; r < n; ++r) tb.K[i][r] = (float)Km[(size_t)r * kL + i];
        for (int k = 0; k < kL; ++k)
            for (int r = 0; r < n; ++r) tb.G[k][r] = (float)Gm[(size_t)k * n + r];
    };
    bool use_modal = false;
    if (modal_ok) {
        auto transform = [&](std::vector<ld> &Km, std::vector<ld> &Gm) {
            Km.assign((size_t)n * kL, 0);
            Gm.assign((size_t)kL * n, 0);
            for (int r = 0; r < n; ++r)
                for (int i = 0; i < kL; ++i) {
                    ld acc = 0;
                    for (int c = 0; c < n; ++c) acc += Winv[(size_t)r * n + c] * Kf[(size_t)c * kL + i];
                    Km[(size_t)r * kL + i] = acc;
                }
            for (int k = 0; k < kL; ++k)
                for (int c = 0; c < n; ++c) {
                    ld acc = 0;
                    for (int r = 0; r < n; ++r) acc += Gf[(size_t)k * n + r] * W[(size_t)r * n + c];
                    Gm[(size_t)k * n + c] = acc;
                }
        };
        std::vector<ld> Km, Gm;
        transform(Km, Gm);
        // balance each slot: equal largest entries in its K rows and G columns
        for (int s = 0; s < S; ++s) {
            ld nk = 0, ng = 0;
            for (int rr = 2 * s; rr < 2 * s + 2; ++rr)
                for (int i = 0; i < kL; ++i) nk = std::max(nk, std::fabs(Km[(size_t)rr * kL + i]));
            for (int k = 0; k < kL; ++k)
                for (int c = 2 * s; c < 2 * s + 2; ++c) ng = std::max(ng, std::fabs(Gm[(size_t)k * n + c]));
            if (nk > 0 && ng > 0) {
                ld sig = std::sqrt(nk / ng);
                for (int r = 0; r < n; ++r) {
                    W[(size_t)r * n + 2 * s] *= sig;
                    W[(size_t)r * n + 2 * s + 1] *= sig;
                }
                for (int c = 0; c < n; ++c) {
                    Winv[(size_t)(2 * s) * n + c] /= sig;
                    Winv[(size_t)(2 * s + 1) * n + c] /= sig;
                }
            }
        }
        transform(Km, Gm);
        pl->kappa = (double)(frob(W) * frob(Winv));
        fill_tables(Km, Gm);
        double ML[kMaxSlots][4];
        pl->slot_power(kL, ML);
        for (int s = 0; s < kMaxSlots; ++s)
            for (int q = 0; q < 4; ++q) tb.M[s][q] = (float)ML[s][q];
        pl->probe_err = std::max(probe_modal(*pl, secs, false), probe_modal(*pl, secs, true));
        use_modal = precision == FILARK_PREC_MODAL32 ||
                    ((precision == FILARK_PREC_AUTO || precision == FILARK_PREC_ALL32) && pl->probe_err < 2e-6);
    } else {
        pl->kappa = std::numeric_limits<double>::infinity();
    }
    if (use_modal) {
        pl->W = W;
        pl->Winv = Winv;
        pl->dense = false;
        pl->mode = precision == FILARK_PREC_ALL32 ? FILARK_PREC_ALL32 : FILARK_PREC_MODAL32;
        return FILARK_OK;
    }
    if (precision != FILARK_PREC_AUTO && precision != FILARK_PREC_DENSE64 && precision != FILARK_PREC_ALL32) {
        *err = "unknown precision mode";
        return FILARK_EINVAL;
    }
    // dense carry in the canonical basis (W = I)
    pl->dense = true;
    pl->mode = precision == FILARK_PREC_ALL32 ? FILARK_PREC_ALL32 : FILARK_PREC_DENSE64;
    pl->W.assign((size_t)n * n, 0);
    pl->Winv.assign((size_t)n * n, 0);
    for (int i = 0; i < n; ++i) pl->W[(size_t)i * n + i] = pl->Winv[(size_t)i * n + i] = 1;
    fill_tables(Kf, Gf);
    if (!dense_lane_layout(dense_matrices(A, n), pl->NS, pl->dense_mats)) {
        *err = "dense carry: a transition power is not block lower triangular";
        return FILARK_EINVAL;
    }
    pl->probe_err = probe_dense(*pl, secs, A);
    return FILARK_OK;
}

// ---------------------------------------------------------------------------
// Butterworth bandpass by the bilinear transform.
// ---------------------------------------------------------------------------
filark_status design_butter_bandpass(int order, double f1, double f2, double fs, double *sos,
                                     std::string *err) {
    if (!sos || order < 1 || order > 64 || !(fs > 0) || !(f1 > 0) || !(f2 > f1) || !(f2 < fs / 2)) {
        *err = "butter_bandpass: need order >= 1 and 0 < f1 < f2 < fs/2";
        return FILARK_EINVAL;
    }
    const ld pi = 3.141592653589793238462643383279502884L;
    const ld c = 2 * (ld)fs;                    // bilinear constant 2/T
    const ld w1 = c * std::tan(pi * (ld)f1 / (ld)fs);
    const ld w2 = c * std::tan(pi * (ld)f2 / (ld)fs);
    const ld bw = w2 - w1, w0sq = w1 * w2;
    struct Den { ld a1, a2, radius; };
    std::vector<Den> dens;
    std::vector<ld> reals;
    for (int k = 1; k <= order; ++k) {
        ld t = pi * (ld)(2 * k - 1) / (ld)(2 * order);
        cld p(-std::sin(t), std::cos(t));            // lowpass prototype pole
        cld pb = p * bw;
        cld root = std::sqrt(pb * pb - 4 * w0sq);
        for (cld sp : {(pb + root) / (ld)2, (pb - root) / (ld)2}) {
            cld z = (c + sp) / (c - sp);
            ld tol = 1e-12L * (1 + std::abs(z));
            if (z.imag() > tol)
                dens.push_back({-2 * z.real(), std::norm(z), std::abs(z)});
            else if (std::fabs(z.imag()) <= tol)
                reals.push_back(z.real());
        }
    }
    std::sort(reals.begin(), reals.end());
    for (size_t i = 0; i + 1 < reals.size(); i += 2)
        dens.push_back({-(reals[i] + reals[i + 1]), reals[i] * reals[i + 1],
                        std::max(std::fabs(reals[i]), std::fabs(reals[i + 1]))});
    if ((int)dens.size() != order) {
        *err = "butter_bandpass: pole grouping failed";
        return FILARK_EINVAL;
    }
    std::stable_sort(dens.begin(), dens.end(), [](const Den &a, const Den &b) { return a.radius < b.radius; });
    // Zeros: N at z = +1 and N at z = -1.  The half of the sections with the
    // lowest pole frequencies get (1 - z^-1)^2, the upper half (1 + z^-1)^2,
    // a middle section (odd N) gets 1 - z^-2: each double zero faces the poles
    // it sits next to, which keeps section states small for poles near z = 1.
    std::vector<ld> freq((size_t)order);
    for (int s = 0; s < order; ++s) {
        const ld a1 = dens[(size_t)s].a1, a2 = dens[(size_t)s].a2;
        const ld disc = a1 * a1 - 4 * a2;
        freq[(size_t)s] = disc < 0 ? std::atan2(std::sqrt(-disc), -a1) : (a1 > 0 ? pi : (ld)0);
    }
    std::vector<int> idx((size_t)order);
    for (int s = 0; s < order; ++s) idx[(size_t)s] = s;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return freq[(size_t)a] < freq[(size_t)b]; });
    std::vector<std::array<ld, 3>> num((size_t)order);
    for (int rank = 0; rank < order; ++rank) {
        const int s = idx[(size_t)rank];
        if (rank < order / 2) num[(size_t)s] = {1, -2, 1};
        else if (order % 2 == 1 && rank == order / 2) num[(size_t)s] = {1, 0, -1};
        else num[(size_t)s] = {1, 2, 1};
    }
    const ld wc = 2 * std::atan(std::sqrt(w0sq) / c);
    const cld zc = std::polar((ld)1, -wc);
    cld H = 1;
    for (int s = 0; s < order; ++s) {
        const Den &d = dens[(size_t)s];
        const auto &b = num[(size_t)s];
        H *= (b[0] + b[1] * zc + b[2] * zc * zc) / ((ld)1 + d.a1 * zc + d.a2 * zc * zc);
    }
    const ld g = std::pow(1 / std::abs(H), (ld)1 / (ld)order);
    for (int s = 0; s < order; ++s) {
        for (int q = 0; q < 3; ++q) sos[6 * s + q] = (double)(g * num[(size_t)s][(size_t)q]);
        sos[6 * s + 3] = 1.0;
        sos[6 * s + 4] = (double)dens[(size_t)s].a1;
        sos[6 * s + 5] = (double)dens[(size_t)s].a2;
    }
    return FILARK_OK;
}

void set_unit_geometry(const Plan &plan, int Tl, int nbc, ChainUnit &u) {
    u.T = Tl;
    u.nblk = (Tl + kL - 1) / kL;
    u.Lr = Tl - (u.nblk - 1) * kL;
    u.nbc = nbc;
    u.R = (u.nblk + nbc - 1) / nbc;
    if (plan.NS > 0) {
        const int nb_last = u.nblk - (u.R - 1) * nbc;
        const double (*pl)[4] = plan.power_cached((nb_last - 1) * kL + u.Lr);
        const double (*pr)[4] = plan.power_cached(u.Lr);
        const double (*pp)[4] = plan.power_cached_cta(nbc, u.R - 1);
        for (int s = 0; s < kMaxSlots; ++s) {
            // PhiTot = PhiLast * Phi^(R-1) (2x2 per slot)
            const double *a = pl[s], *b = pp[s];
            const double tot[4] = {a[0] * b[0] + a[1] * b[2], a[0] * b[1] + a[1] * b[3],
                                   a[2] * b[0] + a[3] * b[2], a[2] * b[1] + a[3] * b[3]};
            for (int q = 0; q < 4; ++q) {
                u.Mr32[s][q] = (float)pr[s][q];
                u.PhiLastHi[s][q] = (float)pl[s][q];
                u.PhiLastLo[s][q] = (float)(pl[s][q] - (double)u.PhiLastHi[s][q]);
                u.PhiTotHi[s][q] = (float)tot[q];
                u.PhiTotLo[s][q] = (float)(tot[q] - (double)u.PhiTotHi[s][q]);
            }
        }
    }
}

void set_static_params(const Plan &plan, int hw, int HP, int Wout, int ns, int nl, const float *dense_dev,
                       ChainParams &p) {
    std::memset(&p, 0, sizeof(p));
    p.tab = plan.tab;
    set_cta_powers(plan, kNB, p);
    p.hw = hw;
    p.HP = HP;
    p.Wout = Wout;
    p.ns = ns;
    p.nl = nl;
    p.ratio_scale = (nl > 0 && ns > 0) ? (float)((double)nl / (double)ns) : 0.f;
    p.all32 = plan.mode == FILARK_PREC_ALL32;
    p.dense = dense_dev;
}

void set_cta_powers(const Plan &plan, int nbc, ChainParams &p) {
    for (int r = 0; r < kMaxCluster; ++r) {
        const double (*pr)[4] = plan.power_cached_cta(nbc, r);
        for (int s = 0; s < kMaxSlots; ++s)
            for (int q = 0; q < 4; ++q) p.PhiPow32[r][s][q] = (float)pr[s][q];
    }
}

}  // namespace filark
