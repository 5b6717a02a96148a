/*
 * CPU oracle for single-channel 2D correlation — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may call
 * this file.  It shares no code, header or constant with the CUDA library.
 *
 * Definition (the 2D convolution benchmark kernel of Sec. 5 "Benchmark
 * kernels", whose tunables are listed in Table 1; the paper states no formula,
 * and the workloads fix it as a "valid" cross-correlation without filter flip
 * or padding):
 *
 *     out[y][x] = sum_{i=0}^{fh-1} sum_{j=0}^{fw-1} in[y+i][x+j] * f[i][j]
 *     for 0 <= y < out_h, 0 <= x < out_w; in has (out_h+fh-1) rows and
 *     (out_w+fw-1) valid columns, stored row-major with a row pitch.
 *
 * Precision: every product of two float32 values is exact in float64 (24+24
 * significant bits), and the sum of <= 4096 such terms in float64 carries a
 * relative error below 1e-12 of S = sum |in*f|, far inside the 1e-5*S
 * tolerance the float32 path is held to.  S is returned beside each output so
 * callers can apply that tolerance per pixel.
 *
 * Plain loops, OpenMP over output rows; nothing is blocked, fused or
 * reordered.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Full output.  out and S are out_h x out_w, row-major, contiguous. */
void oracle_corr2d_f64(const float* in, int64_t in_pitch, int out_w, int out_h,
                       const float* f, int fw, int fh,
                       double* out, double* S, int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int y = 0; y < out_h; ++y) {
        for (int x = 0; x < out_w; ++x) {
            double s = 0.0, a = 0.0;
            for (int i = 0; i < fh; ++i) {
                const float* row = in + (int64_t)(y + i) * in_pitch + x;
                for (int j = 0; j < fw; ++j) {
                    double p = (double)row[j] * (double)f[i * fw + j];
                    s += p;
                    a += fabs(p);
                }
            }
            out[(int64_t)y * out_w + x] = s;
            if (S) S[(int64_t)y * out_w + x] = a;
        }
    }
    (void)nthreads;
}

/* The same definition evaluated at n given points (xs[k], ys[k]) only. */
void oracle_corr2d_f64_points(const float* in, int64_t in_pitch,
                              const float* f, int fw, int fh,
                              const int64_t* xs, const int64_t* ys, int64_t n,
                              double* out, double* S)
{
    for (int64_t k = 0; k < n; ++k) {
        double s = 0.0, a = 0.0;
        for (int i = 0; i < fh; ++i) {
            const float* row = in + (ys[k] + i) * in_pitch + xs[k];
            for (int j = 0; j < fw; ++j) {
                double p = (double)row[j] * (double)f[i * fw + j];
                s += p;
                a += fabs(p);
            }
        }
        out[k] = s;
        if (S) S[k] = a;
    }
}

/* BF16 storage reading: a bf16 value is the top 16 bits of a float32, so it
 * widens to float32 (and then to float64) exactly.  in and f hold raw bf16
 * bit patterns; everything else is as above. */
static double bf16_to_f64(uint16_t h)
{
    union { uint32_t u; float f; } v;
    v.u = (uint32_t)h << 16;
    return (double)v.f;
}

void oracle_corr2d_bf16_f64(const uint16_t* in, int64_t in_pitch, int out_w, int out_h,
                            const uint16_t* f, int fw, int fh,
                            double* out, double* S, int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int y = 0; y < out_h; ++y) {
        for (int x = 0; x < out_w; ++x) {
            double s = 0.0, a = 0.0;
            for (int i = 0; i < fh; ++i) {
                const uint16_t* row = in + (int64_t)(y + i) * in_pitch + x;
                for (int j = 0; j < fw; ++j) {
                    double p = bf16_to_f64(row[j]) * bf16_to_f64(f[i * fw + j]);
                    s += p;
                    a += fabs(p);
                }
            }
            out[(int64_t)y * out_w + x] = s;
            if (S) S[(int64_t)y * out_w + x] = a;
        }
    }
    (void)nthreads;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
