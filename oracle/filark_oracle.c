/*
 * filark_oracle.c -- plain, slow, sequential CPU oracle of the chunked DAS
 * operator chain (causal IIR bandpass as second-order sections, spatial
 * moving average, STA/LTA detector), and of the SOS adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * Arithmetic type: `real` (double by default).  The same source is compiled a
 * second time with ORA_LONG_DOUBLE defined, which makes `real` long double and
 * renames every exported symbol from ora_* to orald_*; the tests use that build
 * to bound the rounding error of the double build.
 *
 * What is computed, and which passage of the paper each part follows:
 *   - Streaming contract (Sec. 3.4, stateful-compatible operators; Sec. 6.2):
 *     a chain object carries the full operator state between calls, and the
 *     concatenation of the outputs of any sequence of pushes equals the output
 *     of one push of the whole recording.  Outputs have the input's length.
 *     The state after reset is zero (x[n<0] = y[n<0] = 0), which is what gives
 *     the first chunk the start-up transient that Sec. 6.2 describes.
 *   - IIR stage (Table 1, "IIR ... second-order sections, SOS", realtime
 *     variant): each section in transposed direct form II with a0-normalised
 *     coefficients, sections applied in array order.
 *   - Butterworth bandpass design (the filter the chain is configured with):
 *     analog prototype poles, bilinear transform with prewarped band edges,
 *     conjugate-pair sections whose double zeros face their poles (z = +1 for
 *     the low half, z = -1 for the high half), unit gain at the geometric
 *     band centre.
 *   - Spatial running mean (Table 1, "Spatial ... running mean"; Sec. 3.4,
 *     halo expansion across neighbouring channels): the mean over the channels
 *     c-h..c+h that exist (the window shrinks at the ends of the array).
 *   - Energy detector (Sec. 3.4, threshold-based energy detectors behind the
 *     monitor interface): classic STA/LTA of cf = y^2 with trailing windows that
 *     end at the current sample; the ratio is 0 until the long window is full
 *     and wherever the long window holds only zeros.
 *   - Adjoint of the SOS cascade (gradients with respect to the input and to
 *     every coefficient of every section), for the differentiable filter.
 *   - Stateful temporal operators of the same streaming contract (Table 1,
 *     temporal filters and amplitude operators): a realtime FIR with its input
 *     history carried across pushes (overlap-save), a running mean and a
 *     running AGC over a trailing window, and an EMA power equalisation.
 *   - Trigger and event extraction on the detector ratio (Sec. 3.4, threshold
 *     detectors behind the monitor interface): a per-channel on/off
 *     hysteresis state carried across pushes; every maximal run of the "on"
 *     state is a channel trigger [t_on, t_off); triggers on neighbouring
 *     channels whose time intervals overlap belong to the same event.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORA_LONG_DOUBLE
typedef long double real;
#define ORA(name) orald_##name
#define R_SQRT sqrtl
#define R_FABS fabsl
#define R_SIN sinl
#define R_COS cosl
#define R_TAN tanl
#define R_ATAN atanl
#define R_POW powl
#define R_ATAN2 atan2l
#else
typedef double real;
#define ORA(name) ora_##name
#define R_SQRT sqrt
#define R_FABS fabs
#define R_SIN sin
#define R_COS cos
#define R_TAN tan
#define R_ATAN atan
#define R_POW pow
#define R_ATAN2 atan2
#endif

/* ------------------------------------------------------------------------- */
/* Small complex helpers (kept explicit so every step is visible).            */
/* ------------------------------------------------------------------------- */
typedef struct { real re, im; } cplx;

static cplx c_make(real re, real im) { cplx z = {re, im}; return z; }
static cplx c_add(cplx a, cplx b) { return c_make(a.re + b.re, a.im + b.im); }
static cplx c_sub(cplx a, cplx b) { return c_make(a.re - b.re, a.im - b.im); }
static cplx c_mul(cplx a, cplx b) {
    return c_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
static cplx c_div(cplx a, cplx b) {
    real d = b.re * b.re + b.im * b.im;
    return c_make((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
static cplx c_scale(cplx a, real s) { return c_make(a.re * s, a.im * s); }
static real c_abs(cplx a) { return R_SQRT(a.re * a.re + a.im * a.im); }
/* principal square root */
static cplx c_sqrt(cplx a) {
    real r = c_abs(a);
    real re = R_SQRT((r + a.re) / 2);
    real im = R_SQRT((r - a.re) / 2);
    if (a.im < 0) im = -im;
    return c_make(re, im);
}

/* ------------------------------------------------------------------------- */
/* Butterworth bandpass design by the bilinear transform.                     */
/*                                                                            */
/* order N is the order of the analog lowpass prototype; the bandpass has     */
/* order 2N and is returned as N second-order sections, row s being           */
/* {b0, b1, b2, a0, a1, a2} with a0 = 1.                                      */
/* Returns 0 on success, -1 on invalid arguments.                             */
/* ------------------------------------------------------------------------- */
int ORA(butter_bandpass)(int N, double f1, double f2, double fs, double *sos)
{
    if (N < 1 || N > 64 || !(fs > 0) || !(f1 > 0) || !(f2 > f1) || !(f2 < fs / 2) || !sos)
        return -1;
    const real pi = (real)3.14159265358979323846264338327950288L;
    const real two_fs = 2 * (real)fs;
    /* prewarped analog band edges */
    const real W1 = two_fs * R_TAN(pi * (real)f1 / (real)fs);
    const real W2 = two_fs * R_TAN(pi * (real)f2 / (real)fs);
    const real W0sq = W1 * W2;          /* squared geometric centre */
    const real Bw = W2 - W1;            /* bandwidth */

    /* 2N digital poles; keep the ones in the upper half plane (one per
       conjugate pair) and collect real poles separately. */
    cplx *up = (cplx *)malloc(sizeof(cplx) * (size_t)(2 * N));
    real *rp = (real *)malloc(sizeof(real) * (size_t)(2 * N));
    int nup = 0, nrp = 0;
    for (int k = 1; k <= N; ++k) {
        /* analog lowpass prototype pole on the unit circle, left half plane */
        real ang = pi * (real)(2 * k + N - 1) / (real)(2 * N);
        cplx p = c_make(R_COS(ang), R_SIN(ang));
        /* lowpass -> bandpass: s^2 - p*B*s + W0^2 = 0 */
        cplx half = c_scale(p, Bw / 2);
        cplx disc = c_sqrt(c_sub(c_mul(half, half), c_make(W0sq, 0)));
        cplx s_pair[2] = { c_add(half, disc), c_sub(half, disc) };
        for (int q = 0; q < 2; ++q) {
            cplx s = s_pair[q];
            /* bilinear transform z = (2fs + s) / (2fs - s) */
            cplx z = c_div(c_add(c_make(two_fs, 0), s), c_sub(c_make(two_fs, 0), s));
            real tol = 1e-12L * (c_abs(z) + 1);
            if (z.im > tol) up[nup++] = z;
            else if (R_FABS(z.im) <= tol) rp[nrp++] = z.re;
            /* poles with z.im < -tol are the conjugates of kept ones */
        }
    }
    if (nup + nrp / 2 != N || (nrp % 2) != 0) { free(up); free(rp); return -1; }

    /* denominators: conjugate pairs, then real poles paired in order */
    real *rad = (real *)malloc(sizeof(real) * (size_t)N);
    real (*den)[3] = (real (*)[3])malloc(sizeof(real[3]) * (size_t)N);
    int ns = 0;
    for (int i = 0; i < nup; ++i, ++ns) {
        den[ns][0] = 1;
        den[ns][1] = -2 * up[i].re;
        den[ns][2] = up[i].re * up[i].re + up[i].im * up[i].im;
        rad[ns] = c_abs(up[i]);
    }
    for (int i = 0; i + 1 < nrp; i += 2, ++ns) {
        den[ns][0] = 1;
        den[ns][1] = -(rp[i] + rp[i + 1]);
        den[ns][2] = rp[i] * rp[i + 1];
        rad[ns] = R_FABS(rp[i]) > R_FABS(rp[i + 1]) ? R_FABS(rp[i]) : R_FABS(rp[i + 1]);
    }
    /* order sections by ascending pole radius (stable insertion sort) */
    for (int i = 1; i < N; ++i) {
        for (int j = i; j > 0 && rad[j - 1] > rad[j]; --j) {
            real tr = rad[j]; rad[j] = rad[j - 1]; rad[j - 1] = tr;
            for (int q = 0; q < 3; ++q) { real t = den[j][q]; den[j][q] = den[j - 1][q]; den[j - 1][q] = t; }
        }
    }
    /* numerators: the bandpass has N zeros at z = +1 (from s = 0) and N at
       z = -1 (from s = infinity).  The N/2 sections whose poles have the
       lowest frequency (smallest pole angle) take both zeros at z = +1,
       b = (1, -2, 1); the N/2 highest take both at z = -1, b = (1, 2, 1); for
       odd N the middle section takes one of each, b = (1, 0, -1).  Keeping the
       zeros next to the poles they face keeps the TDF-II states of sections
       with poles near z = 1 small (the transfer function is the same for any
       pairing). */
    real (*num)[3] = (real (*)[3])malloc(sizeof(real[3]) * (size_t)N);
    real *ang = (real *)malloc(sizeof(real) * (size_t)N);
    for (int s = 0; s < N; ++s) {
        /* largest |angle| of the section's two poles z^2 + a1 z + a2 = 0 */
        real disc = den[s][1] * den[s][1] - 4 * den[s][2];
        ang[s] = disc < 0 ? R_ATAN2(R_SQRT(-disc), -den[s][1]) : (-den[s][1] < 0 ? (real)3.14159265358979323846264338327950288L : 0);
    }
    for (int s = 0; s < N; ++s) {
        int rank = 0;            /* sections with a strictly smaller angle, ties by index */
        for (int t = 0; t < N; ++t)
            if (ang[t] < ang[s] || (ang[t] == ang[s] && t < s)) ++rank;
        if (rank < N / 2) { num[s][0] = 1; num[s][1] = -2; num[s][2] = 1; }
        else if ((N % 2) == 1 && rank == N / 2) { num[s][0] = 1; num[s][1] = 0; num[s][2] = -1; }
        else { num[s][0] = 1; num[s][1] = 2; num[s][2] = 1; }
    }
    /* gain: |H(e^{j w0})| = 1 at the digital image of the geometric centre,
       spread equally over the sections. */
    const real w0 = 2 * R_ATAN(R_SQRT(W0sq) / two_fs);
    cplx zi = c_make(R_COS(w0), -R_SIN(w0));     /* z^-1 at w0 */
    cplx zi2 = c_mul(zi, zi);
    cplx H = c_make(1, 0);
    for (int s = 0; s < N; ++s) {
        cplx nn = c_add(c_add(c_make(num[s][0], 0), c_scale(zi, num[s][1])), c_scale(zi2, num[s][2]));
        cplx dd = c_add(c_add(c_make(den[s][0], 0), c_scale(zi, den[s][1])), c_scale(zi2, den[s][2]));
        H = c_mul(H, c_div(nn, dd));
    }
    real g = R_POW(1 / c_abs(H), (real)1 / (real)N);
    for (int s = 0; s < N; ++s) {
        sos[6 * s + 0] = (double)(g * num[s][0]);
        sos[6 * s + 1] = (double)(g * num[s][1]);
        sos[6 * s + 2] = (double)(g * num[s][2]);
        sos[6 * s + 3] = (double)den[s][0];
        sos[6 * s + 4] = (double)den[s][1];
        sos[6 * s + 5] = (double)den[s][2];
    }
    free(num); free(ang);
    free(up); free(rp); free(rad); free(den);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* One SOS cascade in transposed direct form II (Table 1, realtime SOS).      */
/*                                                                            */
/* Per section, with coefficients divided by a0:                              */
/*     y  = b0*u + z1                                                         */
/*     z1 = b1*u - a1*y + z2                                                  */
/*     z2 = b2*u - a2*y                                                       */
/* and the output of section s is the input of section s+1.  z holds S*2      */
/* values (z1, z2 per section) and is updated in place, so successive calls   */
/* continue the same stream.                                                  */
/* ------------------------------------------------------------------------- */
static real sos_step(const real *c /* S*5 normalised b0 b1 b2 a1 a2 */, int S, real *z, real u)
{
    for (int s = 0; s < S; ++s) {
        const real *k = c + 5 * s;
        real *zs = z + 2 * s;
        real y = k[0] * u + zs[0];
        zs[0] = k[1] * u - k[3] * y + zs[1];
        zs[1] = k[2] * u - k[4] * y;
        u = y;
    }
    return u;
}

static void normalise_sos(const double *sos, int S, real *c)
{
    for (int s = 0; s < S; ++s) {
        real a0 = (real)sos[6 * s + 3];
        c[5 * s + 0] = (real)sos[6 * s + 0] / a0;
        c[5 * s + 1] = (real)sos[6 * s + 1] / a0;
        c[5 * s + 2] = (real)sos[6 * s + 2] / a0;
        c[5 * s + 3] = (real)sos[6 * s + 4] / a0;
        c[5 * s + 4] = (real)sos[6 * s + 5] / a0;
    }
}

/* Filter one channel: x[0..N) -> y[0..N), state z (S*2, in/out, may be NULL
   for a zero initial state that is discarded afterwards). */
void ORA(sosfilt)(const double *sos, int S, const double *x, long N, double *y, double *z_io)
{
    real *c = (real *)malloc(sizeof(real) * (size_t)(5 * (S > 0 ? S : 1)));
    real *z = (real *)calloc((size_t)(2 * (S > 0 ? S : 1)), sizeof(real));
    normalise_sos(sos, S, c);
    if (z_io) for (int i = 0; i < 2 * S; ++i) z[i] = (real)z_io[i];
    for (long n = 0; n < N; ++n) y[n] = (double)sos_step(c, S, z, (real)x[n]);
    if (z_io) for (int i = 0; i < 2 * S; ++i) z_io[i] = (double)z[i];
    free(c); free(z);
}

/* ------------------------------------------------------------------------- */
/* The chain: IIR -> spatial mean -> STA/LTA, with carried state.             */
/* ------------------------------------------------------------------------- */
typedef struct {
    int C, S, K, ns, nl;
    real *coef;        /* S*5 normalised coefficients */
    real *z;           /* C * S * 2 IIR state */
    real *hist;        /* C * nl: cf[m] for the last nl samples, slot m mod nl */
    real *sta, *lta;   /* C running window sums */
    long *nz;          /* C: count of nonzero cf values in the long window */
    long n;            /* samples since reset */
    long since_resum;  /* samples since the running sums were re-added */
    real *row_bp;      /* C scratch */
} ora_chain_t;

#define RESUM_PERIOD 65536L

void *ORA(chain_new)(int C, int S, const double *sos, int K, int ns, int nl)
{
    if (C < 1 || S < 0 || K < 1 || (K % 2) == 0) return NULL;
    if (ns < 0 || nl < 0 || ns > nl || (ns == 0) != (nl == 0)) return NULL;
    ora_chain_t *h = (ora_chain_t *)calloc(1, sizeof(ora_chain_t));
    h->C = C; h->S = S; h->K = K; h->ns = ns; h->nl = nl;
    h->coef = (real *)calloc((size_t)(5 * (S > 0 ? S : 1)), sizeof(real));
    normalise_sos(sos, S, h->coef);
    h->z = (real *)calloc((size_t)C * (size_t)(2 * (S > 0 ? S : 1)), sizeof(real));
    h->hist = (real *)calloc((size_t)C * (size_t)(nl > 0 ? nl : 1), sizeof(real));
    h->sta = (real *)calloc((size_t)C, sizeof(real));
    h->lta = (real *)calloc((size_t)C, sizeof(real));
    h->nz = (long *)calloc((size_t)C, sizeof(long));
    h->row_bp = (real *)calloc((size_t)C, sizeof(real));
    return h;
}

void ORA(chain_free)(void *p)
{
    ora_chain_t *h = (ora_chain_t *)p;
    if (!h) return;
    free(h->coef); free(h->z); free(h->hist); free(h->sta); free(h->lta);
    free(h->nz); free(h->row_bp); free(h);
}

void ORA(chain_reset)(void *p)
{
    ora_chain_t *h = (ora_chain_t *)p;
    int S2 = 2 * (h->S > 0 ? h->S : 1);
    memset(h->z, 0, sizeof(real) * (size_t)h->C * (size_t)S2);
    memset(h->hist, 0, sizeof(real) * (size_t)h->C * (size_t)(h->nl > 0 ? h->nl : 1));
    memset(h->sta, 0, sizeof(real) * (size_t)h->C);
    memset(h->lta, 0, sizeof(real) * (size_t)h->C);
    memset(h->nz, 0, sizeof(long) * (size_t)h->C);
    h->n = 0; h->since_resum = 0;
}

long ORA(chain_samples)(void *p) { return ((ora_chain_t *)p)->n; }

/* cf value of sample m (m >= 0, within the last nl samples) of channel c */
static real hist_at(const ora_chain_t *h, int c, long m)
{
    return h->hist[(size_t)c * (size_t)h->nl + (size_t)(m % h->nl)];
}

/*
 * Push T samples.  x is time-major: sample t of channel c at x[t*ldx + c].
 * Outputs (time-major, row stride ldo, any may be NULL):
 *   bp    = bandpass output y_bp
 *   sp    = spatial mean y_sp
 *   ratio = STA/LTA (only when the detector is on)
 * Returns 0, or -1 on invalid arguments.
 */
int ORA(chain_push)(void *p, const float *x, long ldx, long T,
                    double *bp, double *sp, double *ratio, long ldo)
{
    ora_chain_t *h = (ora_chain_t *)p;
    if (!h || T < 0 || (T > 0 && !x) || ldx < h->C || ldo < h->C) return -1;
    const int C = h->C, S = h->S, hw = (h->K - 1) / 2;
    const int S2 = 2 * (S > 0 ? S : 1);
    for (long t = 0; t < T; ++t) {
        const long n = h->n;
        /* 1. IIR per channel */
        for (int c = 0; c < C; ++c) {
            real u = (real)x[t * ldx + c];
            h->row_bp[c] = sos_step(h->coef, S, h->z + (size_t)c * (size_t)S2, u);
            if (bp) bp[t * ldo + c] = (double)h->row_bp[c];
        }
        /* 2. spatial mean over the existing channels c-hw..c+hw */
        for (int c = 0; c < C; ++c) {
            int lo = c - hw < 0 ? 0 : c - hw;
            int hi = c + hw > C - 1 ? C - 1 : c + hw;
            real acc = 0;
            for (int q = lo; q <= hi; ++q) acc += h->row_bp[q];
            real ysp = acc / (real)(hi - lo + 1);
            if (sp) sp[t * ldo + c] = (double)ysp;
            /* 3. STA/LTA on cf = ysp^2 */
            if (h->nl > 0) {
                real cf = ysp * ysp;
                real out_s = (n - h->ns >= 0) ? hist_at(h, c, n - h->ns) : 0;
                real out_l = (n - h->nl >= 0) ? hist_at(h, c, n - h->nl) : 0;
                h->sta[c] += cf - out_s;
                h->lta[c] += cf - out_l;
                h->nz[c] += (cf != 0) - (out_l != 0);
                h->hist[(size_t)c * (size_t)h->nl + (size_t)(n % h->nl)] = cf;
                if (ratio) {
                    real r = 0;
                    if (n >= h->nl - 1 && h->nz[c] > 0)
                        r = (h->sta[c] / (real)h->ns) / (h->lta[c] / (real)h->nl);
                    ratio[t * ldo + c] = (double)r;
                }
            }
        }
        h->n += 1;
        /* re-add the windows from the history to bound running-sum drift */
        if (h->nl > 0 && ++h->since_resum >= RESUM_PERIOD) {
            h->since_resum = 0;
            for (int c = 0; c < C; ++c) {
                real s = 0, l = 0;
                for (long m = h->n - h->ns; m < h->n; ++m) if (m >= 0) s += hist_at(h, c, m);
                for (long m = h->n - h->nl; m < h->n; ++m) if (m >= 0) l += hist_at(h, c, m);
                h->sta[c] = s; h->lta[c] = l;
            }
        }
    }
    return 0;
}

/* Export / import the IIR state of every channel in the canonical layout
   (channel-major, per section z1 then z2), so tests can compare states. */
void ORA(chain_get_iir_state)(void *p, double *out)
{
    ora_chain_t *h = (ora_chain_t *)p;
    int S2 = 2 * h->S;
    for (int c = 0; c < h->C; ++c)
        for (int i = 0; i < S2; ++i)
            out[(size_t)c * (size_t)S2 + (size_t)i] = (double)h->z[(size_t)c * (size_t)(S2 > 0 ? S2 : 2) + (size_t)i];
}

/* ------------------------------------------------------------------------- */
/* Literal STA/LTA windows, O(window) per sample, for one channel.            */
/* STA[n] = (1/ns) * sum_{k=n-ns+1..n} cf[k],  LTA likewise with nl,           */
/* cf[k] = 0 for k < 0;  R[n] = STA/LTA if n >= nl-1 and LTA > 0, else 0.     */
/* ------------------------------------------------------------------------- */
void ORA(stalta_naive)(const double *cf, long N, int ns, int nl, double *R)
{
    for (long n = 0; n < N; ++n) {
        real s = 0, l = 0;
        for (long k = n - ns + 1; k <= n; ++k) if (k >= 0) s += (real)cf[k];
        for (long k = n - nl + 1; k <= n; ++k) if (k >= 0) l += (real)cf[k];
        real sta = s / (real)ns, lta = l / (real)nl;
        R[n] = (n >= nl - 1 && lta > 0) ? (double)(sta / lta) : 0.0;
    }
}

/* ------------------------------------------------------------------------- */
/* Adjoint of the SOS cascade for one channel.                                */
/*                                                                            */
/* Section s maps u -> y with a0*y[n] + a1*y[n-1] + a2*y[n-2]                 */
/*                         = b0*u[n] + b1*u[n-1] + b2*u[n-2],                 */
/* zero initial conditions.  Given gy = dL/dy of the cascade output, the      */
/* section's adjoint signal w solves, backwards in time,                      */
/*     a0*w[n] + a1*w[n+1] + a2*w[n+2] = gy[n],  w[n >= N] = 0,               */
/* and then                                                                   */
/*     dL/db_i = sum_n w[n] * u[n-i]                                          */
/*     dL/da_i = -sum_n w[n] * y[n-i]        (i = 0, 1, 2)                    */
/*     dL/du[n] = sum_i b_i * w[n+i]                                          */
/* where the last line is the gy of the previous section.  The forward        */
/* signals of every section are recomputed here from x.                       */
/* gsos (S*6, accumulated into) gets dL/d{b0,b1,b2,a0,a1,a2} per section;     */
/* gx (N) gets dL/dx.                                                         */
/* ------------------------------------------------------------------------- */
void ORA(sos_adjoint)(const double *sos, int S, const double *x, long N,
                      const double *gy_in, double *gx, double *gsos)
{
    real *sig = (real *)malloc(sizeof(real) * (size_t)(S + 1) * (size_t)(N > 0 ? N : 1));
    real *g = (real *)malloc(sizeof(real) * (size_t)(N > 0 ? N : 1));
    real *w = (real *)malloc(sizeof(real) * (size_t)(N > 0 ? N : 1));
    /* forward: sig[s] is the input of section s, sig[S] the cascade output */
    for (long n = 0; n < N; ++n) sig[n] = (real)x[n];
    for (int s = 0; s < S; ++s) {
        const double *k = sos + 6 * s;
        real a0 = (real)k[3];
        real *u = sig + (size_t)s * (size_t)N, *y = sig + (size_t)(s + 1) * (size_t)N;
        for (long n = 0; n < N; ++n) {
            real acc = (real)k[0] * u[n];
            if (n >= 1) acc += (real)k[1] * u[n - 1] - (real)k[4] * y[n - 1];
            if (n >= 2) acc += (real)k[2] * u[n - 2] - (real)k[5] * y[n - 2];
            y[n] = acc / a0;
        }
    }
    for (long n = 0; n < N; ++n) g[n] = (real)gy_in[n];
    for (int s = S - 1; s >= 0; --s) {
        const double *k = sos + 6 * s;
        const real b0 = (real)k[0], b1 = (real)k[1], b2 = (real)k[2];
        const real a0 = (real)k[3], a1 = (real)k[4], a2 = (real)k[5];
        const real *u = sig + (size_t)s * (size_t)N, *y = sig + (size_t)(s + 1) * (size_t)N;
        for (long n = N - 1; n >= 0; --n) {
            real acc = g[n];
            if (n + 1 < N) acc -= a1 * w[n + 1];
            if (n + 2 < N) acc -= a2 * w[n + 2];
            w[n] = acc / a0;
        }
        real gb[3] = {0, 0, 0}, ga[3] = {0, 0, 0};
        for (long n = 0; n < N; ++n) {
            for (int i = 0; i < 3; ++i) {
                if (n - i >= 0) {
                    gb[i] += w[n] * u[n - i];
                    ga[i] -= w[n] * y[n - i];
                }
            }
        }
        gsos[6 * s + 0] += (double)gb[0];
        gsos[6 * s + 1] += (double)gb[1];
        gsos[6 * s + 2] += (double)gb[2];
        gsos[6 * s + 3] += (double)ga[0];
        gsos[6 * s + 4] += (double)ga[1];
        gsos[6 * s + 5] += (double)ga[2];
        /* gradient with respect to this section's input */
        for (long n = 0; n < N; ++n) {
            real acc = b0 * w[n];
            if (n + 1 < N) acc += b1 * w[n + 1];
            if (n + 2 < N) acc += b2 * w[n + 2];
            g[n] = acc;
        }
    }
    for (long n = 0; n < N; ++n) gx[n] = (double)g[n];
    free(sig); free(g); free(w);
}


/* ------------------------------------------------------------------------
 * Triggers (per channel, hysteresis) and events (triggers merged across
 * neighbouring channels).  Integer and comparison work only: the ratio is
 * compared, as given (float), against the double thresholds.
 *
 *   s(-1) = 0;  s(n) = 1 if R(n) >= on,  0 if R(n) < off,  else s(n-1).
 *   A channel trigger is a maximal run of s = 1: [t_on, t_off), t_off the
 *   first sample after the run.  It is reported when the run ends (or, by a
 *   flush, with t_off = samples seen so far and the OPEN flag).
 * ------------------------------------------------------------------------ */
#ifndef ORA_LONG_DOUBLE
typedef struct {
    int C;
    double on, off;
    long n;          /* samples seen */
    int *s;          /* state per channel */
    long *t_open;    /* start of the open run (valid while s = 1) */
} ora_trig_t;

void *ora_trig_new(int C, double on, double off)
{
    ora_trig_t *t = (ora_trig_t *)calloc(1, sizeof(ora_trig_t));
    t->C = C;
    t->on = on;
    t->off = off;
    t->s = (int *)calloc((size_t)C, sizeof(int));
    t->t_open = (long *)calloc((size_t)C, sizeof(long));
    return t;
}

void ora_trig_free(void *p)
{
    ora_trig_t *t = (ora_trig_t *)p;
    if (!t) return;
    free(t->s);
    free(t->t_open);
    free(t);
}

/* One push of T samples of R (time-major, row stride ld).  Appends the
 * triggers that end in this push as (channel, t_on, t_off) to the arrays
 * (at most cap); returns how many ended (which may exceed cap). */
long ora_trig_push(void *p, const float *R, long ld, long T, long *rc, long *ron, long *roff, long cap)
{
    ora_trig_t *t = (ora_trig_t *)p;
    long k = 0;
    for (long i = 0; i < T; ++i) {
        const long n = t->n + i;
        for (int c = 0; c < t->C; ++c) {
            const double r = (double)R[i * ld + c];
            int s = t->s[c];
            if (r >= t->on) s = 1;
            else if (r < t->off) s = 0;
            if (s == 1 && t->s[c] == 0) t->t_open[c] = n;
            if (s == 0 && t->s[c] == 1) {
                if (k < cap) {
                    rc[k] = c;
                    ron[k] = t->t_open[c];
                    roff[k] = n;
                }
                ++k;
            }
            t->s[c] = s;
        }
    }
    t->n += T;
    return k;
}

/* Report the runs still open (t_off = samples seen); the state is kept. */
long ora_trig_flush(void *p, long *rc, long *ron, long *roff, long cap)
{
    ora_trig_t *t = (ora_trig_t *)p;
    long k = 0;
    for (int c = 0; c < t->C; ++c) {
        if (!t->s[c]) continue;
        if (k < cap) {
            rc[k] = c;
            ron[k] = t->t_open[c];
            roff[k] = t->n;
        }
        ++k;
    }
    return k;
}

static long uf_find(long *parent, long i)
{
    while (parent[i] != i) i = parent[i];
    return i;
}

/* Events: connected components of the triggers, two triggers being joined
 * when their channels differ by one and their intervals share a sample.
 * ev receives 5 longs per event {t_on, t_off, c_min, c_max, n_triggers};
 * events are returned sorted by (t_on, c_min, t_off, c_max).  Returns the
 * number of events.  Every pair of triggers is tested (quadratic in n: the
 * plain statement of the rule, kept for its clarity, not its speed). */
static int ev_cmp(const void *a, const void *b)
{
    const long *x = (const long *)a, *y = (const long *)b;
    const int order[4] = {0, 2, 1, 3};
    for (int i = 0; i < 4; ++i) {
        if (x[order[i]] < y[order[i]]) return -1;
        if (x[order[i]] > y[order[i]]) return 1;
    }
    return 0;
}

long ora_events_merge(const long *rc, const long *ron, const long *roff, long n, long *ev)
{
    long *parent = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    long *root_ev = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    for (long i = 0; i < n; ++i) parent[i] = i;
    for (long i = 0; i < n; ++i)
        for (long j = i + 1; j < n; ++j) {
            const long dc = rc[i] - rc[j];
            if (dc != 1 && dc != -1) continue;
            const long lo = ron[i] > ron[j] ? ron[i] : ron[j];
            const long hi = roff[i] < roff[j] ? roff[i] : roff[j];
            if (lo >= hi) continue;
            const long x = uf_find(parent, i), y = uf_find(parent, j);
            if (x != y) parent[x < y ? y : x] = x < y ? x : y;
        }
    long m = 0;
    for (long i = 0; i < n; ++i)
        if (uf_find(parent, i) == i) {
            long *e = ev + 5 * m;
            e[0] = ron[i]; e[1] = roff[i]; e[2] = rc[i]; e[3] = rc[i]; e[4] = 0;
            root_ev[i] = m++;
        }
    for (long j = 0; j < n; ++j) {
        long *e = ev + 5 * root_ev[uf_find(parent, j)];
        if (ron[j] < e[0]) e[0] = ron[j];
        if (roff[j] > e[1]) e[1] = roff[j];
        if (rc[j] < e[2]) e[2] = rc[j];
        if (rc[j] > e[3]) e[3] = rc[j];
        e[4] += 1;
    }
    qsort(ev, (size_t)m, 5 * sizeof(long), ev_cmp);
    free(parent);
    free(root_ev);
    return m;
}
#endif


/* ------------------------------------------------------------------------
 * Temporal operators, per channel, x[n < 0] = 0, state carried across pushes:
 *   FIR      y[n] = sum_{k=0}^{M-1} h[k] x[n-k]
 *   MEAN     y[n] = (1/w) sum_{k=0}^{w-1} x[n-k]
 *   AGC      g[n] = (1/w) sum_{k=0}^{w-1} |x[n-k]|;  y[n] = x[n] / g[n] (0 if g = 0)
 *   EMA      e[n] = (1-a) e[n-1] + a x[n]^2, e[-1] = 0;
 *            y[n] = x[n] / sqrt(e[n]) (0 if e = 0)
 * ------------------------------------------------------------------------ */
#ifndef ORA_LONG_DOUBLE
typedef struct {
    int C, kind, M;     /* kind 0 FIR, 1 MEAN, 2 AGC, 3 EMA; M = taps or window */
    double a;           /* EMA coefficient */
    double *h;          /* FIR taps */
    double *hist;       /* [M][C] last M values of x (FIR, MEAN) or |x| (AGC), ring */
    double *sum;        /* [C] window sums (MEAN, AGC) */
    double *e;          /* [C] EMA state */
    long n;
} ora_top_t;

void *ora_top_new(int C, int kind, int M, const double *h, double a)
{
    ora_top_t *t = (ora_top_t *)calloc(1, sizeof(ora_top_t));
    t->C = C;
    t->kind = kind;
    t->M = M > 0 ? M : 1;
    t->a = a;
    t->h = (double *)calloc((size_t)t->M, sizeof(double));
    if (h) memcpy(t->h, h, sizeof(double) * (size_t)t->M);
    t->hist = (double *)calloc((size_t)t->M * (size_t)C, sizeof(double));
    t->sum = (double *)calloc((size_t)C, sizeof(double));
    t->e = (double *)calloc((size_t)C, sizeof(double));
    return t;
}

void ora_top_free(void *p)
{
    ora_top_t *t = (ora_top_t *)p;
    if (!t) return;
    free(t->h); free(t->hist); free(t->sum); free(t->e);
    free(t);
}

/* value of the history ring for sample m (0 before the stream start) */
static double top_hist(const ora_top_t *t, int c, long m)
{
    if (m < 0) return 0;
    return t->hist[(size_t)(m % t->M) * (size_t)t->C + (size_t)c];
}

void ora_top_push(void *p, const float *x, long ld, long T, double *y, long ldy)
{
    ora_top_t *t = (ora_top_t *)p;
    for (long i = 0; i < T; ++i) {
        const long n = t->n + i;
        for (int c = 0; c < t->C; ++c) {
            const double v = (double)x[i * ld + c];
            double out = 0;
            if (t->kind == 0) {
                /* store first: the k = 0 term is the current sample */
                t->hist[(size_t)(n % t->M) * (size_t)t->C + (size_t)c] = v;
                double acc = 0;
                for (int k = 0; k < t->M; ++k) acc += t->h[k] * top_hist(t, c, n - k);
                out = acc;
            } else if (t->kind == 1 || t->kind == 2) {
                const double u = t->kind == 1 ? v : fabs(v);
                const double old = top_hist(t, c, n - t->M);
                t->hist[(size_t)(n % t->M) * (size_t)t->C + (size_t)c] = u;
                t->sum[c] += u - old;
                if (n % 4096 == 4095) {   /* re-sum the window exactly from time to time */
                    double s = 0;
                    for (long m = n - t->M + 1; m <= n; ++m) s += top_hist(t, c, m);
                    t->sum[c] = s;
                }
                const double g = t->sum[c] / (double)t->M;
                if (t->kind == 1) out = g;
                else out = g > 0 ? v / g : 0;
            } else {
                t->e[c] = (1 - t->a) * t->e[c] + t->a * v * v;
                out = t->e[c] > 0 ? v / sqrt(t->e[c]) : 0;
            }
            y[i * ldy + c] = out;
        }
    }
    t->n += T;
}
#endif
