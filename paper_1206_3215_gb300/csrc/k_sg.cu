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
#include "sg_sin.cuh"

namespace pss {

template <class Rl> __device__ __forceinline__ Rl sin_(Rl a) { return sg_sin(a); }
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
    static constexpr bool EARLY_NEXT = true;
    V2<Rl> *h;  // in: H rows; out: S rows (in place)
    __device__ const V2<Rl> *in(int) const { return h; }
    template <int N, int P, int BLOCK, class Sm, class H = NoHook>
    __device__ __forceinline__ void row(V2<Rl> (&vv)[1][P], int64_t r, bool ok, int t, const Sm (&sm)[1],
                                        const TW<Rl> *tw, const H &hook = H{}) const
    {
        V2<Rl>(&v)[P] = vv[0];
        if constexpr (sg_shared(sizeof(Rl))) {
            conj_all(v);
#pragma unroll 1
            for (int pass = 0; pass < 2; ++pass) {
                block_fft<N, P, -1, BLOCK>(v, sm[0], t, tw, [&]() {
                    if (pass == 1) hook();
                });
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
            block_fft<N, P, -1, BLOCK>(v, sm[0], t, tw, hook);
        }
        store_line<P, N / P>(v, h + r * N, 1, t, ok);
    }
};

template <class Rl> struct SgCol {
    static constexpr int NIN = 1;
    // not COL_LAND: the landing-buffer column pass was slower for this op
    // (2048^2 FP32 half spectra 86.6 -> 77.2 Gpt-steps/s, full 48.7 -> 44.5)
    static constexpr bool LEAN = sg_shared(sizeof(Rl));
    static constexpr int PMAX = 32;
    V2<Rl> *h;          // in: S columns; out: next H
    V2<Rl> *u, *d;      // uhat^n, d^n, updated in place
    const Rl *kx2, *ky2;
    Rl dt2, inv_n2;     // dt^2, 1/(nx ny)
    int64_t nx;
    int *status;        // set when a tile copy did not arrive
    __host__ __device__ const V2<Rl> *in(int) const { return h; }
    template <int N, int P, int BLOCK, class Sm>
    __device__ __forceinline__ void col(V2<Rl> (&vv)[1][P], int64_t field, int x, int t,
                                        const Sm (&sm)[1], const TW<Rl> *tw) const
    {
        constexpr int T = N / P;
        V2<Rl>(&v)[P] = vv[0];
        const int64_t base = field * N * nx + x;
        const int64_t step = int64_t(T) * nx;
        {
            // u and d are read only after the forward transform: have them in L2 by then
            const V2<Rl> *qu = u + base + int64_t(t) * nx, *qd = d + base + int64_t(t) * nx;
#pragma unroll
            for (int m = 0; m < P; ++m, qu += step, qd += step) {
                prefetch_l2(qu);
                prefetch_l2(qd);
            }
        }
        auto update = [&]() {
            const Rl kx = __ldg(kx2 + x);
            // û and d of point m + LA are loaded while point m is computed and
            // stored: the loads are placed before the earlier points' stores
            // in program order (the compiler keeps loads and stores that may
            // alias in that order; û, d and h are separate arrays and every
            // point is its own row, so they do not alias), so LA points are
            // always in flight instead of waiting one round trip per chunk
            constexpr int LA = P < 4 ? P : 4;
            const V2<Rl> *lu = u + base + int64_t(t) * nx, *ld = d + base + int64_t(t) * nx;
            V2<Rl> *su = u + base + int64_t(t) * nx, *sd = d + base + int64_t(t) * nx;
            V2<Rl> ru[LA], rd[LA];
#pragma unroll
            for (int j = 0; j < LA; ++j, lu += step, ld += step) {
                ru[j] = ld_stream(lu);
                rd[j] = ld_stream(ld);
            }
#pragma unroll
            for (int m = 0; m < P; ++m, su += step, sd += step) {
                const V2<Rl> un = ru[m % LA], dn = rd[m % LA];
                if (m + LA < P) {
                    ru[m % LA] = ld_stream(lu);
                    rd[m % LA] = ld_stream(ld);
                    lu += step;
                    ld += step;
                }
                const int y = t + T * m;
                const Rl a = dt2 * (kx + __ldg(ky2 + y));
                const Rl inv = rcp_(Rl(1) + Rl(0.25) * a);
                const V2<Rl> dn1{dn.x - (a * un.x + dt2 * v[m].x) * inv, dn.y - (a * un.y + dt2 * v[m].y) * inv};
                const V2<Rl> un1{un.x + dn1.x, un.y + dn1.y};
                *sd = dn1;
                *su = un1;
                v[m] = cscale(un1, inv_n2);
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

// nx: row stride of the arrays (the columns processed); nreal: points per
// row of the real-space field (nx for full spectra, more for half spectra)
template <class Rl>
cudaError_t sg_col_pass(V2<Rl> *h, V2<Rl> *u, V2<Rl> *d, int64_t nx, int64_t ny, int64_t batch,
                        const Rl *kx2, const Rl *ky2, Rl dt, const TW<Rl> *twy, int *status, cudaStream_t s,
                        int64_t nreal)
{
    SgCol<Rl> op{h, u, d, kx2, ky2, dt * dt, Rl(1.0 / (double(nreal > 0 ? nreal : nx) * double(ny))), nx, status};
    return launch_col<Rl>(ny, nx, op, twy, batch, s);
}

#define PSS_INST(Rl)                                                                              \
    template cudaError_t sg_row_pass<Rl>(V2<Rl> *, int64_t, int64_t, const TW<Rl> *, cudaStream_t); \
    template cudaError_t sg_col_pass<Rl>(V2<Rl> *, V2<Rl> *, V2<Rl> *, int64_t, int64_t, int64_t,   \
                                         const Rl *, const Rl *, Rl, const TW<Rl> *, int *, cudaStream_t, \
                                         int64_t);
PSS_INST(float)
PSS_INST(double)

}  // namespace pss
