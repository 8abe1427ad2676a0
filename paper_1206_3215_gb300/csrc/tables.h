// Host-side tables, computed in FP64 and rounded once to the working precision.
#pragma once
#include <stdint.h>

#include <vector>

namespace pss {

// (cos, sin) of 2 pi e / n, with the angle reduced to the first octant in
// exact integer arithmetic before calling libm.
void cis_2pi(int64_t e, int64_t n, double *c, double *s);

// wavenumber of storage index m: 2 pi / L * m for m < n/2, 2 pi / L * (m - n) otherwise
double wavenumber(int64_t m, int64_t n, double L);

// FP32 pair within one unit in the last place of (c, s) per component whose
// squared modulus is closest to 1 (ties: nearest to (c, s)).
void unit_pair_f32(double c, double s, float *fc, float *fs);

// (re, im) as FP32 hi + lo: out4 = {hi.re, hi.im, lo.re, lo.im}, hi the
// nearest float and lo the rounded residual.
void hilo_f32(double re, double im, float *out4);

// Twiddle table W_n^e = exp(-2 pi i e / n), e = 0..n-1: FP32 as hi + lo
// quadruples (4 floats per entry), FP64 as (re, im) pairs.
std::vector<float> twiddles_f32(int64_t n);
std::vector<double> twiddles_f64(int64_t n);

}  // namespace pss
