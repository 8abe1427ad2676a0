// Host-side table generation in FP64.
#include "tables.h"

#include <cmath>

namespace pss {

static const double kHalfPi = 1.57079632679489661923132169163975144;

void cis_2pi(int64_t e, int64_t n, double *c, double *s)
{
    e %= n;
    if (e < 0) e += n;
    // 2 pi e / n = (pi/2) (q + r/n), q = quadrant, 0 <= r < n
    const int64_t q = (4 * e) / n, r = 4 * e - q * n;
    double cr, sr;
    if (2 * r <= n) {
        const double a = kHalfPi * double(r) / double(n);
        cr = std::cos(a);
        sr = std::sin(a);
    } else {
        const double a = kHalfPi * double(n - r) / double(n);
        cr = std::sin(a);
        sr = std::cos(a);
    }
    switch (q) {
    case 0: *c = cr; *s = sr; break;
    case 1: *c = -sr; *s = cr; break;
    case 2: *c = -cr; *s = -sr; break;
    default: *c = sr; *s = -cr; break;
    }
}

double wavenumber(int64_t m, int64_t n, double L)
{
    const int64_t ms = (m < n / 2) ? m : m - n;
    return 4.0 * kHalfPi / L * double(ms);
}

static double ulp_f32(double x)
{
    const float f = float(std::fabs(x));
    return double(std::nextafter(f, INFINITY)) - double(f);
}

void unit_pair_f32(double c, double s, float *fc, float *fs)
{
    const float c0 = float(c), s0 = float(s);
    float bc = c0, bs = s0;
    double berr = std::fabs(double(c0) * c0 + double(s0) * s0 - 1.0);
    double bdist = std::fabs(double(c0) - c) + std::fabs(double(s0) - s);
    const double uc = ulp_f32(c), us = ulp_f32(s);
    for (int dc = -1; dc <= 1; ++dc)
        for (int ds = -1; ds <= 1; ++ds) {
            float cc = c0, ss = s0;
            if (dc) cc = std::nextafter(c0, dc > 0 ? INFINITY : -INFINITY);
            if (ds) ss = std::nextafter(s0, ds > 0 ? INFINITY : -INFINITY);
            if (std::fabs(double(cc) - c) > uc || std::fabs(double(ss) - s) > us) continue;
            if (std::fabs(cc) > 1.0f || std::fabs(ss) > 1.0f) continue;
            const double err = std::fabs(double(cc) * cc + double(ss) * ss - 1.0);
            const double dist = std::fabs(double(cc) - c) + std::fabs(double(ss) - s);
            if (err < berr || (err == berr && dist < bdist)) {
                bc = cc;
                bs = ss;
                berr = err;
                bdist = dist;
            }
        }
    *fc = bc;
    *fs = bs;
}

void hilo_f32(double re, double im, float *out4)
{
    out4[0] = float(re);
    out4[1] = float(im);
    out4[2] = float(re - double(out4[0]));
    out4[3] = float(im - double(out4[1]));
}

std::vector<float> twiddles_f32(int64_t n)
{
    std::vector<float> t(4 * size_t(n));
    for (int64_t e = 0; e < n; ++e) {
        double c, s;
        cis_2pi(e, n, &c, &s);
        hilo_f32(c, -s, &t[4 * e]);
    }
    return t;
}

std::vector<double> twiddles_f64(int64_t n)
{
    std::vector<double> t(2 * size_t(n));
    for (int64_t e = 0; e < n; ++e) {
        double c, s;
        cis_2pi(e, n, &c, &s);
        t[2 * e] = c;
        t[2 * e + 1] = -s;
    }
    return t;
}

}  // namespace pss
