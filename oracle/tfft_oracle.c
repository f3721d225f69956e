/*
 * tfft_oracle.c -- plain FP64 CPU reference for the batched 1-D C2C FFT.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load it.  It shares no code, header, table
 * or constant with the CUDA library and includes nothing from it.
 *
 * What it computes (TurboFFT, Section II, the DFT definition):
 *     forward  y_j = sum_n x_n exp(-2 pi i j n / N)          (unnormalised)
 *     inverse  x_j = (1/N) sum_n y_n exp(+2 pi i j n / N)
 * The fast path here is the textbook iterative radix-2 decimation-in-time
 * Cooley-Tukey FFT with an explicit bit-reversal permutation -- deliberately
 * NOT the Stockham autosort form the GPU uses, so a shared indexing mistake
 * cannot cancel out.  Twiddles are cos/sin of 2*pi*m/N with the integer m
 * reduced exactly to the first octant before any floating point is involved.
 *
 * Data layout: interleaved (re, im) doubles, signal-major [batch][n].
 * Errors: every entry point returns 0 on success and -1 on a bad argument
 * (n not a power of two, n < 1, batch < 0, null pointer).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

static int is_pow2(int64_t n) { return n >= 1 && (n & (n - 1)) == 0; }

/* exp(sign * 2 pi i m / n) for integer m, reduced exactly to an octant. */
static void unit_root(int64_t m, int64_t n, int sign, double *c, double *s)
{
    const double quarter_pi = 0.78539816339744830961566084581987572;
    int64_t t = m % n;
    if (t < 0) t += n;
    int64_t a = 8 * t;               /* angle = (pi/4) * a / n */
    int64_t q = a / n;               /* octant 0..7 */
    int64_t rem = a - q * n;         /* 0 <= rem < n */
    double cc, ss;
    if ((q & 1) == 0) {
        double phi = quarter_pi * ((double)rem / (double)n);
        double c0 = cos(phi), s0 = sin(phi);
        switch (q) {
        case 0: cc = c0;  ss = s0;  break;
        case 2: cc = -s0; ss = c0;  break;
        case 4: cc = -c0; ss = -s0; break;
        default: cc = s0; ss = -c0; break; /* q == 6 */
        }
    } else {
        double phi = quarter_pi * ((double)(n - rem) / (double)n);
        double c1 = cos(phi), s1 = sin(phi);
        switch (q) {
        case 1: cc = s1;  ss = c1;  break;  /* pi/2 - phi  */
        case 3: cc = -c1; ss = s1;  break;  /* pi - phi    */
        case 5: cc = -s1; ss = -c1; break;  /* 3pi/2 - phi */
        default: cc = c1; ss = -s1; break;  /* 2pi - phi, q == 7 */
        }
    }
    *c = cc;
    *s = (sign < 0) ? -ss : ss;
}

static void bit_reverse(double *z, int64_t n)
{
    int64_t j = 0;
    for (int64_t i = 0; i < n - 1; i++) {
        if (i < j) {
            double tr = z[2 * i], ti = z[2 * i + 1];
            z[2 * i] = z[2 * j]; z[2 * i + 1] = z[2 * j + 1];
            z[2 * j] = tr; z[2 * j + 1] = ti;
        }
        int64_t k = n >> 1;
        while (k >= 1 && (j & k)) { j ^= k; k >>= 1; }
        j |= k;
    }
}

/* One signal, in place, radix-2 DIT, FP64.  sign = -1 forward, +1 inverse
 * (the inverse is NOT scaled here; the caller divides by n).  Each stage
 * first tabulates its len/2 twiddles, then sweeps the array once, so a stage
 * streams through memory once even when the signal is far larger than cache. */
static int fft_one(double *z, int64_t n, int sign)
{
    if (n == 1) return 0;
    double *tw = (double *)malloc(sizeof(double) * n);   /* up to n/2 complex */
    if (!tw) return -1;
    bit_reverse(z, n);
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t half = len >> 1;
        for (int64_t k = 0; k < half; k++) unit_root(k, len, sign, &tw[2 * k], &tw[2 * k + 1]);
        for (int64_t i = 0; i < n; i += len) {
            for (int64_t k = 0; k < half; k++) {
                double wr = tw[2 * k], wi = tw[2 * k + 1];
                double *a = z + 2 * (i + k), *b = z + 2 * (i + k + half);
                double vr = b[0] * wr - b[1] * wi;
                double vi = b[0] * wi + b[1] * wr;
                b[0] = a[0] - vr; b[1] = a[1] - vi;
                a[0] = a[0] + vr; a[1] = a[1] + vi;
            }
        }
    }
    free(tw);
    return 0;
}

/* Forward (sign=-1) or inverse (sign=+1, scaled by 1/n) transform of `batch`
 * signals of length n, in place on interleaved doubles. */
int oracle_fft(double *z, int64_t n, int64_t batch, int sign)
{
    if (!z || !is_pow2(n) || batch < 0 || (sign != 1 && sign != -1)) return -1;
    for (int64_t b = 0; b < batch; b++) {
        double *s = z + 2 * n * b;
        if (fft_one(s, n, sign) != 0) return -1;
        if (sign > 0) {
            double inv = 1.0 / (double)n;
            for (int64_t i = 0; i < 2 * n; i++) s[i] *= inv;
        }
    }
    return 0;
}

/* Brute-force O(n^2) DFT in long double (any n >= 1, not only powers of
 * two), out of place: the direct sum of the definition.  Used only to pin
 * oracle_fft on small sizes. */
int oracle_dft_naive(const double *x, double *y, int64_t n, int64_t batch, int sign)
{
    if (!x || !y || n < 1 || batch < 0 || (sign != 1 && sign != -1)) return -1;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int64_t b = 0; b < batch; b++) {
        const double *xs = x + 2 * n * b;
        double *ys = y + 2 * n * b;
        for (int64_t j = 0; j < n; j++) {
            long double ar = 0.0L, ai = 0.0L;
            for (int64_t k = 0; k < n; k++) {
                int64_t m = (j * k) % n;
                long double ang = (long double)sign * two_pi * (long double)m / (long double)n;
                long double c = cosl(ang), s = sinl(ang);
                ar += (long double)xs[2 * k] * c - (long double)xs[2 * k + 1] * s;
                ai += (long double)xs[2 * k] * s + (long double)xs[2 * k + 1] * c;
            }
            if (sign > 0) { ar /= (long double)n; ai /= (long double)n; }
            ys[2 * j] = (double)ar;
            ys[2 * j + 1] = (double)ai;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Fault emulation (Section II-A fault model: one soft error in a compute unit,
 * realised as one flipped bit of one intermediate value).
 *
 * Runs the same radix-2 DIT forward transform of ONE signal, in FP32
 * (prec == 32: every add/mul rounded to float, twiddles rounded from FP64)
 * or FP64 (prec == 64), and after stage `stage` flips bit `bit` of the real
 * (comp == 0) or imaginary (comp == 1) part of element `elem` of the working
 * array.  stage == -1 corrupts the input value after it is loaded and
 * permuted; stage == log2(n)-1 corrupts an output value.  The result is
 * written as doubles to y.  bit < 0 disables the flip (a clean FP32/FP64 run).
 * ---------------------------------------------------------------------- */
static void flip_f32(float *v, int bit)
{
    uint32_t u; memcpy(&u, v, 4); u ^= (uint32_t)1u << bit; memcpy(v, &u, 4);
}
static void flip_f64(double *v, int bit)
{
    uint64_t u; memcpy(&u, v, 8); u ^= (uint64_t)1u << bit; memcpy(v, &u, 8);
}

int oracle_fft_faulty(const double *x, double *y, int64_t n, int prec,
                      int stage, int64_t elem, int comp, int bit)
{
    if (!x || !y || !is_pow2(n) || (prec != 32 && prec != 64)) return -1;
    int log2n = 0; while ((INT64_C(1) << log2n) < n) log2n++;
    if (bit >= 0) {
        if (stage < -1 || stage >= log2n || elem < 0 || elem >= n || comp < 0 || comp > 1) return -1;
        if (bit >= prec) return -1;
    }
    if (prec == 64) {
        double *z = (double *)malloc(sizeof(double) * 2 * n);
        if (!z) return -1;
        memcpy(z, x, sizeof(double) * 2 * n);
        bit_reverse(z, n);
        if (bit >= 0 && stage == -1) flip_f64(&z[2 * elem + comp], bit);
        int s = 0;
        for (int64_t len = 2; len <= n; len <<= 1, s++) {
            int64_t half = len >> 1;
            for (int64_t k = 0; k < half; k++) {
                double wr, wi; unit_root(k, len, -1, &wr, &wi);
                for (int64_t i = 0; i < n; i += len) {
                    double *a = z + 2 * (i + k), *b = z + 2 * (i + k + half);
                    double vr = b[0] * wr - b[1] * wi, vi = b[0] * wi + b[1] * wr;
                    b[0] = a[0] - vr; b[1] = a[1] - vi;
                    a[0] = a[0] + vr; a[1] = a[1] + vi;
                }
            }
            if (bit >= 0 && stage == s) flip_f64(&z[2 * elem + comp], bit);
        }
        memcpy(y, z, sizeof(double) * 2 * n);
        free(z);
    } else {
        float *z = (float *)malloc(sizeof(float) * 2 * n);
        if (!z) return -1;
        for (int64_t i = 0; i < 2 * n; i++) z[i] = (float)x[i];
        /* bit reversal on floats */
        int64_t j = 0;
        for (int64_t i = 0; i < n - 1; i++) {
            if (i < j) {
                float tr = z[2 * i], ti = z[2 * i + 1];
                z[2 * i] = z[2 * j]; z[2 * i + 1] = z[2 * j + 1];
                z[2 * j] = tr; z[2 * j + 1] = ti;
            }
            int64_t k = n >> 1;
            while (k >= 1 && (j & k)) { j ^= k; k >>= 1; }
            j |= k;
        }
        if (bit >= 0 && stage == -1) flip_f32(&z[2 * elem + comp], bit);
        int s = 0;
        for (int64_t len = 2; len <= n; len <<= 1, s++) {
            int64_t half = len >> 1;
            for (int64_t k = 0; k < half; k++) {
                double wr64, wi64; unit_root(k, len, -1, &wr64, &wi64);
                float wr = (float)wr64, wi = (float)wi64;
                for (int64_t i = 0; i < n; i += len) {
                    float *a = z + 2 * (i + k), *b = z + 2 * (i + k + half);
                    float t0 = b[0] * wr, t1 = b[1] * wi, t2 = b[0] * wi, t3 = b[1] * wr;
                    float vr = t0 - t1, vi = t2 + t3;
                    float ar = a[0], ai = a[1];
                    b[0] = ar - vr; b[1] = ai - vi;
                    a[0] = ar + vr; a[1] = ai + vi;
                }
            }
            if (bit >= 0 && stage == s) flip_f32(&z[2 * elem + comp], bit);
        }
        for (int64_t i = 0; i < 2 * n; i++) y[i] = (double)z[i];
        free(z);
    }
    return 0;
}
