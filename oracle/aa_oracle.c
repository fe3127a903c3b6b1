/*
 * aa_oracle.c -- plain CPU oracle for brute-force incoherent dedispersion and
 * the single-pulse search (boxcar SNR + thresholded local-maximum peaks).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  It is used by tests/, by __graft_entry__.smoke() and by the
 * cpu_baseline / reference legs of bench.py, and nowhere else.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * Every function is the textbook definition written out as scalar loops:
 * FP64 for frequencies, delays, mean, standard deviation and SNR; exact int64
 * for every sum of samples.  The paper (arXiv:1912.07704) names the modules
 * (dedispersion, boxcar single-pulse search with peak finding, Sec. 1) and the
 * pipeline shape (Sec. 2.3-3.3); the arithmetic below is the brute-force
 * method it refers to:
 *
 *   f_c     = fch1 + c*foff                              (channel centre, MHz)
 *   f_top   = highest channel frequency
 *   Delta_c = f_c^-2 - f_top^-2
 *   DM_i    = dm_lo + i*dm_step                          (not accumulated)
 *   s(c,i)  = round_half_away(((K*DM_i)*Delta_c) / (tsamp*dec)),  K = 4.148808e3
 *   x_r[c][j] = sum_{k<dec} x[c][j*dec+k],  j < floor(T/dec)
 *   y[i][t]   = sum_c x_r[c][t + s(c,i)],   t < L = floor(T/dec) - max s
 *   mu, sigma = population mean / std of y[i][0..L)  (optionally of the
 *               samples kept by iterative k-sigma clipping, see below)
 *   SNR_w(t)  = (sum_{k<w} y[t+k] - w*mu) / (sigma*sqrt(w)),  1 <= w <= min(W, L-t)
 *   B(t)      = max_w SNR_w(t)  (smallest w on ties)
 *   peak at t iff B(t) >= thr and B(t) > B(t-1) and B(t) >= B(t+1)
 *                 (missing neighbours count as -infinity; sigma == 0 rows
 *                  have B = 0 and no peaks)
 *
 * Compile with -ffp-contract=off so that every FP64 operation is rounded
 * separately, in the order written.  OpenMP (when enabled) only splits
 * independent outputs across threads; integer sums do not depend on order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_K_DM 4.148808e3 /* MHz^2 pc^-1 cm^3 s */

int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Highest channel frequency: fch1 when foff < 0, the last channel otherwise. */
double oracle_f_top(double fch1, double foff, int32_t nchans)
{
    double f_last = fch1 + (double)(nchans - 1) * foff;
    return f_last > fch1 ? f_last : fch1;
}

/* Integer delay of every channel for one DM, in samples of the decimated
 * series.  Returns how many channels fell within 1e-9 of a half-integer
 * (where the rounding direction is decided by the last bits). */
int32_t oracle_shifts(int32_t nchans, double fch1, double foff, double tsamp,
                      double dm, int32_t dec, int32_t* out)
{
    double ft = oracle_f_top(fch1, foff, nchans);
    int32_t near_half = 0;
    for (int32_t c = 0; c < nchans; ++c) {
        double fc = fch1 + (double)c * foff;
        double delta = 1.0 / (fc * fc) - 1.0 / (ft * ft);
        double v = ORACLE_K_DM * dm * delta / (tsamp * (double)dec);
        if (fabs(v - floor(v) - 0.5) < 1e-9) near_half++;
        out[c] = (int32_t)llround(v);
    }
    return near_half;
}

/* Sub-band dedispersion (an approximation of the brute-force sum): channels
 * in bands of `band` consecutive channels, each with a reference channel, its
 * highest frequency (the band's first channel when foff < 0, else its last).
 * Delay of every channel relative to its band's reference at one DM, in
 * decimated samples: round half away of ((K*dm)*(delta_c - delta_ref)) /
 * (tsamp*dec), delta as in oracle_shifts. */
void oracle_subband_rel(int32_t nchans, double fch1, double foff, double tsamp, double dm,
                        int32_t dec, int32_t band, int32_t* out)
{
    double ft = oracle_f_top(fch1, foff, nchans);
    for (int32_t c = 0; c < nchans; ++c) {
        int32_t b0 = (c / band) * band;
        int32_t b1 = b0 + band - 1 < nchans - 1 ? b0 + band - 1 : nchans - 1;
        int32_t cr = foff < 0 ? b0 : b1;
        double fc = fch1 + (double)c * foff;
        double fr = fch1 + (double)cr * foff;
        double dc = 1.0 / (fc * fc) - 1.0 / (ft * ft);
        double dr = 1.0 / (fr * fr) - 1.0 / (ft * ft);
        out[c] = (int32_t)llround(ORACLE_K_DM * dm * (dc - dr) / (tsamp * (double)dec));
    }
}

/* FDMT-style tree dedispersion (an approximation of the brute-force sum:
 * delays are split between subbands, not computed per channel).  Channels
 * are taken in order of delta_c = f_c^-2 - f_top^-2 (falling frequency);
 * dk[k] is the k-th smallest.  A subband [a, b] of that order with delay
 * delta (of its channel b relative to its channel a) is split at
 * m = a + ceil((b - a + 1) / 2) into [a, m-1] with delay
 *   round_half_away(delta * (dk[m-1] - dk[a]) / (dk[b] - dk[a]))
 * and [m, b] starting gap = round_half_away(delta * (dk[m] - dk[a]) /
 * (dk[b] - dk[a])) later, with delay delta - gap; a single channel has
 * delay 0.  e[k] receives the delay of the k-th channel for the whole band's
 * delay delta at offset base. */
static void fdmt_split(const double* dk, int32_t a, int32_t b, int64_t delta, int64_t base, int64_t* e)
{
    if (a == b) {
        e[a] = base;
        return;
    }
    const int32_t m = a + (b - a + 2) / 2;
    const double span = dk[b] - dk[a];
    const int64_t gap = span > 0.0 ? llround((double)delta * (dk[m] - dk[a]) / span) : 0;
    const int64_t du = span > 0.0 ? llround((double)delta * (dk[m - 1] - dk[a]) / span) : 0;
    fdmt_split(dk, a, m - 1, du, base, e);
    fdmt_split(dk, m, b, delta - gap, base + gap, e);
}

/* Effective delay of every channel (channel order, out[c]) when the whole
 * band's delay -- its lowest-frequency channel relative to its highest -- is
 * D samples. */
void oracle_fdmt_delays(int32_t nchans, double fch1, double foff, int64_t D, int32_t* out)
{
    double ft = oracle_f_top(fch1, foff, nchans);
    double* dk = (double*)malloc(sizeof(double) * (size_t)nchans);
    int64_t* e = (int64_t*)malloc(sizeof(int64_t) * (size_t)nchans);
    if (!dk || !e) { free(dk); free(e); return; }
    for (int32_t k = 0; k < nchans; ++k) {
        const int32_t c = foff < 0 ? k : nchans - 1 - k;  /* k-th highest frequency */
        const double fc = fch1 + (double)c * foff;
        dk[k] = 1.0 / (fc * fc) - 1.0 / (ft * ft);
    }
    fdmt_split(dk, 0, nchans - 1, D, 0, e);
    for (int32_t k = 0; k < nchans; ++k) out[foff < 0 ? k : nchans - 1 - k] = (int32_t)e[k];
    free(dk);
    free(e);
}

/* Time decimation by summation; the trailing partial bin is dropped. */
void oracle_decimate(const uint8_t* x, int32_t nchans, int64_t nsamp, int64_t pitch,
                     int32_t dec, uint16_t* out, int64_t out_pitch)
{
    int64_t nd = nsamp / dec;
    for (int32_t c = 0; c < nchans; ++c) {
        for (int64_t j = 0; j < nd; ++j) {
            uint32_t s = 0;
            for (int32_t k = 0; k < dec; ++k) s += x[(int64_t)c * pitch + j * dec + k];
            out[(int64_t)c * out_pitch + j] = (uint16_t)s;
        }
    }
}

static inline int64_t sample_at(const void* x, int32_t elem_bytes, int64_t idx)
{
    if (elem_bytes == 1) return ((const uint8_t*)x)[idx];
    return ((const uint16_t*)x)[idx];
}

/* One dedispersed series y[t] = sum_c x[c][t + shifts[c]] for t in [t0, t1).
 * x is [nchans][pitch] with 1- or 2-byte unsigned samples.  The sum over c is
 * an exact integer sum, so it is taken channel by channel over blocks of
 * consecutive t (each channel's samples read in order); OpenMP splits the
 * blocks. */
void oracle_dedisperse(const void* x, int32_t elem_bytes, int32_t nchans, int64_t pitch,
                       const int32_t* shifts, int64_t t0, int64_t t1, int64_t* out)
{
    const int64_t block = 4096;
    if (t1 - t0 <= 0) return;
#pragma omp parallel for schedule(static)
    for (int64_t b = t0; b < t1; b += block) {
        const int64_t e = b + block < t1 ? b + block : t1;
        for (int64_t t = b; t < e; ++t) out[t - t0] = 0;
        for (int32_t c = 0; c < nchans; ++c) {
            const int64_t row = (int64_t)c * pitch + shifts[c];
            for (int64_t t = b; t < e; ++t) out[t - t0] += sample_at(x, elem_bytes, row + t);
        }
    }
}

/* Population mean and standard deviation of a series (two passes, FP64). */
void oracle_moments(const int64_t* y, int64_t n, double* mu, double* sigma)
{
    if (n <= 0) { *mu = 0.0; *sigma = 0.0; return; }
    int64_t s = 0;
    for (int64_t t = 0; t < n; ++t) s += y[t];
    double m = (double)s / (double)n;
    double ss = 0.0;
    for (int64_t t = 0; t < n; ++t) {
        double d = (double)y[t] - m;
        ss += d * d;
    }
    *mu = m;
    *sigma = sqrt(ss / (double)n);
}

/* Robust mean / standard deviation by iterative k-sigma clipping (outlier
 * rejection for the single-pulse search's statistics), k = c16/16, inclusive
 * bounds, population sigma.  Pass 0 takes every sample; each clipping pass
 * keeps the samples with |y - mu| <= k*sigma of the previous kept set.  With
 * N, S1 = sum y and S2 = sum y^2 of that set, mu = S1/N and
 * sigma = sqrt(N*S2 - S1^2)/N, so (multiplying by 16N and squaring, both
 * sides being >= 0) the test is decided exactly in integers:
 *     256*(N*y - S1)^2 <= c16^2 * (N*S2 - S1^2).
 * At most max_iters clipping passes; a pass that keeps nothing is dropped and
 * ends the iteration; a pass whose kept set has the same (N, S1, S2) as the
 * previous one is a fixed point (the next pass would keep the same set) and
 * ends it too.  mu, sigma: two-pass FP64 over the final kept set. */
void oracle_moments_clipped(const int64_t* y, int64_t n, int32_t c16, int32_t max_iters,
                            double* mu, double* sigma, int64_t* nkept)
{
    *mu = 0.0;
    *sigma = 0.0;
    *nkept = 0;
    if (n <= 0) return;
    unsigned char* keep = (unsigned char*)malloc((size_t)n);
    unsigned char* next = (unsigned char*)malloc((size_t)n);
    if (!keep || !next) { free(keep); free(next); return; }
    __int128 N = 0, S1 = 0, S2 = 0;
    for (int64_t t = 0; t < n; ++t) {
        keep[t] = 1;
        N += 1;
        S1 += y[t];
        S2 += (__int128)y[t] * y[t];
    }
    for (int32_t it = 0; it < max_iters; ++it) {
        const __int128 V = N * S2 - S1 * S1;
        const __int128 R = (__int128)c16 * c16 * V;
        __int128 N2 = 0, T1 = 0, T2 = 0;
        for (int64_t t = 0; t < n; ++t) {
            const __int128 d = N * y[t] - S1;
            next[t] = 256 * d * d <= R;
            if (next[t]) {
                N2 += 1;
                T1 += y[t];
                T2 += (__int128)y[t] * y[t];
            }
        }
        if (N2 == 0) break;
        const int same = N2 == N && T1 == S1 && T2 == S2;
        memcpy(keep, next, (size_t)n);
        N = N2;
        S1 = T1;
        S2 = T2;
        if (same) break;
    }
    int64_t cnt = 0, s = 0;
    for (int64_t t = 0; t < n; ++t)
        if (keep[t]) { ++cnt; s += y[t]; }
    const double m = (double)s / (double)cnt;
    double ss = 0.0;
    for (int64_t t = 0; t < n; ++t)
        if (keep[t]) {
            const double d = (double)y[t] - m;
            ss += d * d;
        }
    *mu = m;
    *sigma = sqrt(ss / (double)cnt);
    *nkept = cnt;
    free(keep);
    free(next);
}

/* Exhaustive boxcar search for t in [t0, t1) of a series of length n.
 * B[t-t0] = max_{1<=w<=min(W,n-t)} SNR_w(t); wbest = smallest maximising w;
 * margin = B minus the best SNR over all other widths (+inf if only one). */
void oracle_boxcar(const int64_t* y, int64_t n, double mu, double sigma, int32_t W,
                   int64_t t0, int64_t t1, double* B, int32_t* wbest, double* margin)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = t0; t < t1; ++t) {
        int64_t k = t - t0;
        if (sigma == 0.0) {
            B[k] = 0.0;
            wbest[k] = 1;
            margin[k] = INFINITY;
            continue;
        }
        int64_t wmax = n - t < (int64_t)W ? n - t : (int64_t)W;
        int64_t S = 0;
        double best = -INFINITY, second = -INFINITY;
        int32_t bw = 0;
        for (int64_t w = 1; w <= wmax; ++w) {
            S += y[t + w - 1];
            double snr = ((double)S - (double)w * mu) / (sigma * sqrt((double)w));
            if (snr > best) {
                second = best;
                best = snr;
                bw = (int32_t)w;
            } else if (snr > second) {
                second = snr;
            }
        }
        B[k] = best;
        wbest[k] = bw;
        margin[k] = best - second;
    }
}

/* oracle_boxcar over a subset of widths: width w (1 <= w <= W) takes part
 * iff wset[w - 1] != 0; B, the smallest maximising width and the margin are
 * those of the widths taking part. */
void oracle_boxcar_widths(const int64_t* y, int64_t n, double mu, double sigma, int32_t W,
                          const uint8_t* wset, int64_t t0, int64_t t1, double* B, int32_t* wbest,
                          double* margin)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = t0; t < t1; ++t) {
        int64_t k = t - t0;
        if (sigma == 0.0) {
            B[k] = 0.0;
            wbest[k] = 1;
            margin[k] = INFINITY;
            continue;
        }
        int64_t wmax = n - t < (int64_t)W ? n - t : (int64_t)W;
        int64_t S = 0;
        double best = -INFINITY, second = -INFINITY;
        int32_t bw = 0;
        for (int64_t w = 1; w <= wmax; ++w) {
            S += y[t + w - 1];
            if (!wset[w - 1]) continue;
            double snr = ((double)S - (double)w * mu) / (sigma * sqrt((double)w));
            if (snr > best) {
                second = best;
                best = snr;
                bw = (int32_t)w;
            } else if (snr > second) {
                second = snr;
            }
        }
        B[k] = best;
        wbest[k] = bw;
        margin[k] = best - second;
    }
}

/* Decimated width ladder (approximate search for wide boxcars: the cited
 * search method, Sec. 1, evaluates wide boxcars on the series decimated by
 * pairs).  Level 0: widths 1..min(W0, W) of the windows starting at t.
 * Level k >= 1 (while W0 * 2^(k-1) < W): widths w = m * 2^k with
 * W0/2 < m <= W0 and w <= W, of the windows starting at the level-k grid
 * point s = floor(t / 2^k) * 2^k <= t, i.e. m consecutive samples of the
 * series decimated k times by pairs; every window inside [0, n).  SNR as in
 * oracle_boxcar; widths are visited in increasing order (level 0, then
 * level 1, ...), so ties go to the smallest width.  B, smallest maximising
 * width and margin as oracle_boxcar; sbest = the start of the maximising
 * window (t, or the grid point of its level).  Returns -1 if the prefix
 * sums cannot be allocated, else 0. */
int oracle_boxcar_dec(const int64_t* y, int64_t n, double mu, double sigma, int32_t W, int32_t W0,
                      int64_t t0, int64_t t1, double* B, int32_t* wbest, double* margin,
                      int64_t* sbest)
{
    int64_t* P = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!P) return -1;
    P[0] = 0;
    for (int64_t i = 0; i < n; ++i) P[i + 1] = P[i] + y[i];
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = t0; t < t1; ++t) {
        int64_t k0 = t - t0;
        if (sigma == 0.0) {
            B[k0] = 0.0;
            wbest[k0] = 1;
            margin[k0] = INFINITY;
            sbest[k0] = t;
            continue;
        }
        double best = -INFINITY, second = -INFINITY;
        int32_t bw = 0;
        int64_t bs = t;
        for (int64_t w = 1; w <= (int64_t)W0 && w <= (int64_t)W && t + w <= n; ++w) {
            double snr = ((double)(P[t + w] - P[t]) - (double)w * mu) / (sigma * sqrt((double)w));
            if (snr > best) {
                second = best;
                best = snr;
                bw = (int32_t)w;
            } else if (snr > second) {
                second = snr;
            }
        }
        for (int k = 1; ((int64_t)W0 << (k - 1)) < (int64_t)W; ++k) {
            int64_t s = (t >> k) << k;
            for (int64_t m = W0 / 2 + 1; m <= W0; ++m) {
                int64_t w = m << k;
                if (w > (int64_t)W || s + w > n) break;
                double snr = ((double)(P[s + w] - P[s]) - (double)w * mu) / (sigma * sqrt((double)w));
                if (snr > best) {
                    second = best;
                    best = snr;
                    bw = (int32_t)w;
                    bs = s;
                } else if (snr > second) {
                    second = snr;
                }
            }
        }
        B[k0] = best;
        wbest[k0] = bw;
        margin[k0] = best - second;
        sbest[k0] = bs;
    }
    free(P);
    return 0;
}

/* Thresholded local maxima of B over [0, n): returns the number found and
 * writes up to cap indices. */
int64_t oracle_peaks(const double* B, int64_t n, double thr, int64_t* out_t, int64_t cap)
{
    int64_t found = 0;
    for (int64_t t = 0; t < n; ++t) {
        double left = t > 0 ? B[t - 1] : -INFINITY;
        double right = t + 1 < n ? B[t + 1] : -INFINITY;
        if (B[t] >= thr && B[t] > left && B[t] >= right) {
            if (found < cap) out_t[found] = t;
            found++;
        }
    }
    return found;
}

/* ---- differentiable (float-weighted) form -------------------------------
 * Forward:  y[d][t] = sum_c w[c] * x[c][t + s(c,d)],  t < L
 * Adjoint (transpose of the forward in x, definition written as a scatter):
 *   gx[c][t + s(c,d)] += w[c] * gy[d][t]
 *   gw[c]             += gy[d][t] * x[c][t + s(c,d)]
 * Loss:     mean over d, t of (y[d][t] - T[d][t])^2
 * All in FP64.
 */
void oracle_forward_f64(const double* x, int32_t nchans, int64_t pitch, const double* w,
                        const int32_t* shifts, int64_t L, double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < L; ++t) {
        double acc = 0.0;
        for (int32_t c = 0; c < nchans; ++c)
            acc += w[c] * x[(int64_t)c * pitch + t + shifts[c]];
        out[t] = acc;
    }
}

/* shifts: [ndm][nchans]; gy: [ndm][L]; gx: [nchans][pitch] (accumulated);
 * gw: [nchans] (accumulated). */
void oracle_adjoint_f64(const double* x, int32_t nchans, int64_t pitch, const double* w,
                        const int32_t* shifts, int32_t ndm, const double* gy, int64_t L,
                        double* gx, double* gw)
{
#pragma omp parallel for schedule(static)
    for (int32_t c = 0; c < nchans; ++c) {
        for (int32_t d = 0; d < ndm; ++d) {
            const int32_t s = shifts[(int64_t)d * nchans + c];
            for (int64_t t = 0; t < L; ++t) {
                const double g = gy[(int64_t)d * L + t];
                gx[(int64_t)c * pitch + t + s] += w[c] * g;
                gw[c] += g * x[(int64_t)c * pitch + t + s];
            }
        }
    }
}
