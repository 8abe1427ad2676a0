// Fused passes of the sine-Gordon semi-implicit leapfrog (Eq. 3, Section 4.2).
//
// The scheme (u^{n+1} - 2u^n + u^{n-1})/dt^2 - Lap (u^{n+1} + 2u^n + u^{n-1})/4
// = -sin u^n is solved in Fourier space.  The two time levels are held as
// uhat^n and the increment d^n = uhat^n - uhat^{n-1}; with a = dt^2 |k|^2 the
// recurrence
//   uhat^{n+1} = [(2 - a/2) uhat^n - dt^2 F sin u^n] / (1 + a/4) - uhat^{n-1}
// is, identically,
//   d^{n+1} = d^n - (a uhat^n + dt^2 F sin u^n) / (1 + a/4),
//   uhat^{n+1} = uhat^n + d^{n+1},
// which forms the small increment directly instead of the difference of two
// nearly equal levels (the cancellation would otherwise cost FP32 most of
// its digits at dt = 1e-3).
//
// State between passes: H = column inverse transform of uhat^n / (nx ny)
// (x in Fourier space, y physical).  A row pass turns H into u^n, takes
// sin u^n and transforms the row forward (S).  A column pass transforms S
// forward (F sin u^n), updates uhat and d in place, and writes the column
// inverse transform of the new uhat as the next H.
#include "launch.cuh"

namespace pss {

// FP32 sin u: Cody-Waite reduction modulo pi/2 and Taylor polynomials on
// [-pi/4, pi/4].  pi/2 = C1 + C2 + C3 (each a float, 72 bits together, from
// the double-double pi/2 below), subtracted with fused multiply-adds, so the
// reduced argument is accurate to a few ulp while |k| < 2^20 (|u| < 1.6e6).
// The omitted Taylor terms r^11/11! and r^12/12! are below 2e-9 on the
// interval.  A non-finite u gives NaN (no loop, no library slow path).
namespace sinc {
constexpr double HI = 1.5707963267948966, LO = 6.123233995736766e-17;  // pi/2 = HI + LO
constexpr float C1 = float(HI);
constexpr float C2 = float(HI - double(C1));
constexpr float C3 = float((HI - double(C1) - double(C2)) + LO);
}  // namespace sinc
#ifndef PSS_SG_LIBM_SIN
#define PSS_SG_LIBM_SIN 0
#endif
__device__ __forceinline__ float sin_(float x)
{
    if constexpr (PSS_SG_LIBM_SIN) return sinf(x);
    const float k = rintf(x * float(2.0 / 3.14159265358979323846));
    float r = __fmaf_rn(-k, sinc::C1, x);
    r = __fmaf_rn(-k, sinc::C2, r);
    r = __fmaf_rn(-k, sinc::C3, r);
    const float r2 = r * r;
    const float sn = __fmaf_rn(r * r2, -1.0f / 6 + r2 * (1.0f / 120 + r2 * (-1.0f / 5040 + r2 * (1.0f / 362880))), r);
    const float cs = 1.0f + r2 * (-0.5f + r2 * (1.0f / 24 + r2 * (-1.0f / 720 + r2 * (1.0f / 40320 + r2 * (-1.0f / 3628800)))));
    const int q = int(k) & 3;
    const float v = (q & 1) ? cs : sn;
    return (q & 2) ? -v : v;
}
__device__ __forceinline__ double sin_(double a) { return sin(a); }
// correctly rounded reciprocal
__device__ __forceinline__ float rcp_(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double rcp_(double a) { return __drcp_rn(a); }

// FP32: both transforms of a pass run through one forward-FFT body
// (F^-1 x = conj(F conj x)), which keeps the pass within 128 registers.
constexpr bool sg_shared(int bytes) { return bytes == 4; }

template <class Rl> struct SgRow {
    static constexpr int NIN = 1;
    static constexpr bool LEAN = sg_shared(sizeof(Rl));
    static constexpr int PMAX = 32;
    V2<Rl> *h;  // in: H rows; out: S rows (in place)
    __device__ const V2<Rl> *in(int) const { return h; }
    template <int N, int P, bool BLOCK, class Sm>
    __device__ __forceinline__ void row(V2<Rl> (&vv)[1][P], int64_t r, bool ok, int t, const Sm (&sm)[1],
                                        const TW<Rl> *tw) const
    {
        V2<Rl>(&v)[P] = vv[0];
        if constexpr (sg_shared(sizeof(Rl))) {
            conj_all(v);
#pragma unroll 1
            for (int pass = 0; pass < 2; ++pass) {
                block_fft<N, P, -1, BLOCK>(v, sm[0], t, tw);
                if (pass == 0)  // u = Re F^-1 H = Re conj(F conj H) = Re F conj H
#pragma unroll
                    for (int m = 0; m < P; ++m) v[m] = V2<Rl>{sin_(v[m].x), Rl(0)};
            }
        } else {
            block_fft<N, P, +1, BLOCK>(v, sm[0], t, tw);
            fence(v);
#pragma unroll
            for (int m = 0; m < P; ++m) v[m] = V2<Rl>{sin_(v[m].x), Rl(0)};
            fence(v);
            block_fft<N, P, -1, BLOCK>(v, sm[0], t, tw);
        }
        store_line<P, N / P>(v, h + r * N, 1, t, ok);
    }
};

template <class Rl> struct SgCol {
    static constexpr int NIN = 1;
    static constexpr bool LEAN = sg_shared(sizeof(Rl));
    static constexpr int PMAX = 32;
    V2<Rl> *h;          // in: S columns; out: next H
    V2<Rl> *u, *d;      // uhat^n, d^n, updated in place
    const Rl *kx2, *ky2;
    Rl dt2, inv_n2;     // dt^2, 1/(nx ny)
    int64_t nx;
    __device__ const V2<Rl> *in(int) const { return h; }
    template <int N, int P, bool BLOCK, class Sm>
    __device__ __forceinline__ void col(V2<Rl> (&vv)[1][P], int64_t field, int x, int t,
                                        const Sm (&sm)[1], const TW<Rl> *tw) const
    {
        constexpr int T = N / P;
        V2<Rl>(&v)[P] = vv[0];
        const int64_t base = field * N * nx + x;
        auto update = [&]() {
            const Rl kx = __ldg(kx2 + x);
            // one running pointer per array (T rows apart), so the 2P loads and
            // stores do not each hold a 64-bit address
            const int64_t step = int64_t(T) * nx;
            V2<Rl> *pu = u + base + int64_t(t) * nx, *pd = d + base + int64_t(t) * nx;
#pragma unroll
            for (int m = 0; m < P; ++m) {
                const int y = t + T * m;
                const V2<Rl> un = *pu, dn = *pd;
                const Rl a = dt2 * (kx + __ldg(ky2 + y));
                const Rl inv = rcp_(Rl(1) + Rl(0.25) * a);
                const V2<Rl> dn1{dn.x - (a * un.x + dt2 * v[m].x) * inv, dn.y - (a * un.y + dt2 * v[m].y) * inv};
                const V2<Rl> un1{un.x + dn1.x, un.y + dn1.y};
                *pd = dn1;
                *pu = un1;
                v[m] = cscale(un1, inv_n2);
                pu += step;
                pd += step;
            }
        };
        if constexpr (sg_shared(sizeof(Rl))) {
#pragma unroll 1
            for (int pass = 0; pass < 2; ++pass) {
                block_fft<N, P, -1, BLOCK>(v, sm[0], t, tw);
                if (pass == 0) {
                    update();
                    conj_all(v);
                }
            }
            conj_all(v);
        } else {
            block_fft<N, P, -1, BLOCK>(v, sm[0], t, tw);
            fence(v);
            update();
            fence(v);
            block_fft<N, P, +1, BLOCK>(v, sm[0], t, tw);
        }
        store_line<P, T>(v, h + base, nx, t, true);
    }
};

template <class Rl>
cudaError_t sg_row_pass(V2<Rl> *h, int64_t nx, int64_t rows_total, const TW<Rl> *twx, cudaStream_t s)
{
    return launch_row<Rl>(nx, SgRow<Rl>{h}, twx, rows_total, s);
}

template <class Rl>
cudaError_t sg_col_pass(V2<Rl> *h, V2<Rl> *u, V2<Rl> *d, int64_t nx, int64_t ny, int64_t batch,
                        const Rl *kx2, const Rl *ky2, Rl dt, const TW<Rl> *twy, cudaStream_t s)
{
    SgCol<Rl> op{h, u, d, kx2, ky2, dt * dt, Rl(1.0 / (double(nx) * double(ny))), nx};
    return launch_col<Rl>(ny, nx, op, twy, batch, s);
}

#define PSS_INST(Rl)                                                                              \
    template cudaError_t sg_row_pass<Rl>(V2<Rl> *, int64_t, int64_t, const TW<Rl> *, cudaStream_t); \
    template cudaError_t sg_col_pass<Rl>(V2<Rl> *, V2<Rl> *, V2<Rl> *, int64_t, int64_t, int64_t,   \
                                         const Rl *, const Rl *, Rl, const TW<Rl> *, cudaStream_t);
PSS_INST(float)
PSS_INST(double)

}  // namespace pss
