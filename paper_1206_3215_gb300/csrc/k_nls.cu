// Fused passes of the NLS split-step Fourier method (Section 4.1).
//
// The state between passes is the row transform of psi.  A row pass takes the
// row inverse transform (giving psi in physical space), applies the exact
// nonlinear sub-step psi <- exp(-i sigma |psi|^2 dt) psi and transforms the row
// forward again.  A column pass transforms the columns forward (giving
// psi_hat), applies the exact linear sub-step psi_hat <- exp(-i |k|^2 tau)
// psi_hat and transforms the columns back.  Each pass reads and writes the
// state once.
#include "launch.cuh"

namespace pss {

// sin(th) and cos(th) - 1 of the nonlinear phase, both without cancellation.
// Taylor series on |a| <= A (FP32: 1/2, FP64: 1/16), where the first omitted
// terms (a^11/11!, a^12/12!) are below 3e-11 (FP32) and 2e-20 (FP64)
// relative to the kept sums.  At the workload's dt |psi|^2 ~ 1e-3 that is the
// whole computation.  A larger phase is first halved k times (exact scaling
// by 2^-k) and then doubled back with
//   sin 2a = 2 sin a (1 + (cos a - 1)),  cos 2a - 1 = 2 (cos a - 1)(cos a - 1 + 2),
// which keeps both terms free of cancellation; k is bounded by the exponent
// range, so a non-finite phase ends in NaN after a bounded loop.
template <class Rl> constexpr Rl phase_taylor_range() { return sizeof(Rl) == 4 ? Rl(0.5) : Rl(0.0625); }

// the Taylor sums alone (|a| within phase_taylor_range)
template <class Rl> __device__ __forceinline__ void phase_taylor(Rl a, Rl &sn, Rl &cm1)
{
    const Rl t2 = a * a;
    sn = a * (Rl(1) + t2 * (Rl(-1.0 / 6) + t2 * (Rl(1.0 / 120) + t2 * (Rl(-1.0 / 5040) + t2 * Rl(1.0 / 362880)))));
    cm1 = t2 * (Rl(-0.5) + t2 * (Rl(1.0 / 24) + t2 * (Rl(-1.0 / 720) + t2 * (Rl(1.0 / 40320) + t2 * Rl(-1.0 / 3628800)))));
}

// FP32 on |a| <= 1/64 (the workload's phases are ~1e-3): sin a = a - a^3/6 and
// cos a - 1 = -a^2/2 + a^4/24, whose first omitted terms (a^5/120, a^6/720)
// are below 1e-11 relative to the unit modulus, far under one FP32 rounding
constexpr float phase_short_range() { return 1.0f / 64; }
__device__ __forceinline__ void phase_short(float a, float &sn, float &cm1)
{
    const float t2 = a * a;
    sn = __fmaf_rn(a * t2, -1.0f / 6, a);
    cm1 = t2 * __fmaf_rn(t2, 1.0f / 24, -0.5f);
}

template <class Rl> __device__ __forceinline__ void phase_terms(Rl th, Rl &sn, Rl &cm1)
{
    constexpr int KMAX = sizeof(Rl) == 4 ? 130 : 1026;
    constexpr Rl A = phase_taylor_range<Rl>();
    Rl a = th;
    int k = 0;
#pragma unroll 1
    while (!(fabs(a) <= A) && k < KMAX) {
        a *= Rl(0.5);
        ++k;
    }
    phase_taylor(a, sn, cm1);
#pragma unroll 1
    for (; k > 0; --k) {
        const Rl s2 = Rl(2) * sn * (Rl(1) + cm1);
        cm1 = Rl(2) * cm1 * (cm1 + Rl(2));
        sn = s2;
    }
}

// FP32 runs both transforms through one forward-FFT body (fewer registers and
// instruction-cache misses); FP64 keeps the two specialised bodies.
#ifndef PSS_SHARED_FFT
#define PSS_SHARED_FFT 1
#endif

template <class Rl> struct NlsRow {
    static constexpr int NIN = 1;
    static constexpr bool LEAN = true;
    static constexpr int PMAX = 32;
    static constexpr bool EARLY_NEXT = true;
    V2<Rl> *data;
    Rl sigma_dt;
    __device__ const V2<Rl> *in(int) const { return data; }
    template <int N, int P, int BLOCK, class Sm, class H = NoHook>
    __device__ __forceinline__ void row(V2<Rl> (&vv)[1][P], int64_t row, bool ok, int t,
                                        const Sm (&smm)[1], const TW<Rl> *tw, const H &hook = H{}) const
    {
        constexpr int T = N / P;
        V2<Rl>(&v)[P] = vv[0];
        const Sm &sm = smm[0];
        V2<Rl> *p = data + row * N;
        auto nonlinear = [&]() {
            // psi exp(-i th) = psi + psi (cos th - 1 - i sin th): the
            // increment is formed without cancellation, so the modulus is
            // kept to the final rounding.  When every phase of this thread is
            // in the Taylor range (always, at the workload's dt |psi|^2), the
            // straight-line Taylor code runs (FP32: the short sums below
            // 1/64); the halving path is out of line.
            Rl big = Rl(0);
#pragma unroll
            for (int m = 0; m < P; ++m) big = fmax(big, fabs(sigma_dt * (v[m].x * v[m].x + v[m].y * v[m].y)));
            auto apply = [&](auto terms) {
#pragma unroll
                for (int m = 0; m < P; ++m) {
                    const Rl x = v[m].x, y = v[m].y;
                    Rl sn, cm1;
                    terms(sigma_dt * (x * x + y * y), sn, cm1);
                    v[m].x = x + (x * cm1 + y * sn);
                    v[m].y = y + (y * cm1 - x * sn);
                }
            };
            // one straight-line body (FP32: the short sums; FP64: the Taylor
            // sums) and the general path, so the code stays small
            bool fast;
            if constexpr (sizeof(Rl) == 4) fast = big <= phase_short_range();
            else fast = big <= phase_taylor_range<Rl>();
            if (fast) {
                apply([](Rl a, Rl &sn, Rl &cm1) {
                    if constexpr (sizeof(Rl) == 4) phase_short(a, sn, cm1);
                    else phase_taylor(a, sn, cm1);
                });
            } else {
#pragma unroll
                for (int m = 0; m < P; ++m) {
                    const Rl x = v[m].x, y = v[m].y;
                    Rl sn, cm1;
                    phase_terms(sigma_dt * (x * x + y * y), sn, cm1);
                    v[m].x = x + (x * cm1 + y * sn);
                    v[m].y = y + (y * cm1 - x * sn);
                }
            }
        };
        if constexpr (PSS_SHARED_FFT && sizeof(Rl) == 4) {
            conj_all(v);
#pragma unroll 1
            for (int pass = 0; pass < 2; ++pass) {
                block_fft<N, P, -1, BLOCK>(v, sm, t, tw, [&]() {
                    if (pass == 1) hook();
                });
                if (pass == 0) {
                    conj_all(v);
                    nonlinear();
                }
            }
        } else {
            block_fft<N, P, +1, BLOCK>(v, sm, t, tw);
            fence(v);
            nonlinear();
            fence(v);
            block_fft<N, P, -1, BLOCK>(v, sm, t, tw, hook);
        }
        store_line<P, T>(v, p, 1, t, ok);
    }
};

// Propagator exp(-i k^2 tau) applied as z + z (K - 1): K - 1 is tabulated
// exactly (hi + lo in FP32) and the small increment z (K - 1) is formed with
// relative accuracy, so each output is one rounding of z + increment.  The
// direct product z K would round x cos + y sin for the slowly rotating low
// wavenumbers in the same direction step after step (K is within a few ulp of
// 1 there), which shows up as a steady drift of the mass in FP32.
template <class V, class W> __device__ __forceinline__ V apply_km1(V z, W km1)
{
    return cadd(z, twmul<-1>(z, km1));
}

// s z + z (s (K - 1)) for a power of two s, given skm1 = s (K - 1) (hi + lo):
// the increment is formed as in apply_km1 and s z (exact) is added inside
// the last fused multiply-add, so the result is bitwise that of
// apply_km1(s z, K - 1) with the scaling folded in (two instructions fewer)
__device__ __forceinline__ float2 apply_skm1(float2 z, float s, float4 skm1)
{
    const float cr = __fmaf_rn(z.x, skm1.z, -z.y * skm1.w);
    const float ci = __fmaf_rn(z.x, skm1.w, z.y * skm1.z);
    const float ir = __fmaf_rn(z.x, skm1.x, __fmaf_rn(-z.y, skm1.y, cr));
    const float ii = __fmaf_rn(z.x, skm1.y, __fmaf_rn(z.y, skm1.x, ci));
    return {__fmaf_rn(z.x, s, ir), __fmaf_rn(z.y, s, ii)};
}

// row factors of the propagator kept in flight per thread (FP32 column pass)
#ifndef PSS_KD
#define PSS_KD 4
#endif

// a 16-byte read-only global load kept in program order
__device__ __forceinline__ float4 ldg_nc_f4(const float4 *p)
{
    float4 r;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
    return r;
}

// The FP32 column pass at n = 1024 keeps the row factors exp(-i ky^2 tau) - 1
// in shared memory: only n/2 + 1 distinct values (ky^2 is even in ky), 8 KB,
// which fits beside every column kernel's buffers without lowering its
// occupancy.  The landing-buffer pass leaves the L1 cache too little room to
// keep the 16 KB table, whose loads then wait on L2.  At other lengths the
// factors are read from the global table.
__host__ __device__ constexpr bool nls_ky_smem(int n) { return n == 1024; }
template <int NH> __device__ __forceinline__ float4 *nls_ky_cache()
{
    __shared__ __align__(16) float4 cache[NH];
    return cache;
}

template <class Rl> struct NlsCol {
    static constexpr int NIN = 1;
    static constexpr bool LEAN = true;
    static constexpr int PMAX = 32;
    // all threads of the CTA, before the first tile: the row factors of
    // ky index 0 .. n/2 into shared memory (the kernel synchronises after)
    template <int N> __device__ __forceinline__ void prologue() const
    {
        if constexpr (sizeof(Rl) == 4 && nls_ky_smem(N)) {
            float4 *c = nls_ky_cache<N / 2 + 1>();
            for (int i = int(threadIdx.x); i <= N / 2; i += int(blockDim.x)) c[i] = __ldg(by + i);
        }
    }
    static constexpr bool COL_LAND = true;  // exchanges sync through fft_sync<BLOCK> only
    // col() takes a hook: the one-buffer pass (4096^2 and larger) issues the
    // next tile's copy at the start of the last stage (column pass 300 -> 279 us
    // at 4096^2, 790 -> 761 us at 8192^2; the SG and NS column ops were slower
    // with it)
    static constexpr bool COL_EARLY = true;
    // in place: the landing-buffer pass stores each tile with one tensor copy
    static constexpr bool COL_TMA_STORE = true;
    V2<Rl> *data;
    int64_t nx;
    Rl scale;
    const TW<Rl> *ax, *by;  // exp(-i kx^2 tau) - 1, exp(-i ky^2 tau) - 1
    int *status;            // set when a tile copy did not arrive
    __host__ __device__ const V2<Rl> *in(int) const { return data; }
    template <int N, int P, int BLOCK, class Sm, class H = NoHook, bool STORE = true>
    __device__ __forceinline__ void col(V2<Rl> (&vv)[1][P], int64_t field, int x, int t,
                                        const Sm (&smm)[1], const TW<Rl> *tw, const H &hook = H{}) const
    {
        constexpr int T = N / P;
        V2<Rl>(&v)[P] = vv[0];
        const Sm &sm = smm[0];
        V2<Rl> *p = data + field * N * nx + x;
        auto propagate = [&]() {
            const TW<Rl> a = __ldg(ax + x);
            const TW<Rl> *byl = launder(by);  // keep these loads after the transform
            if constexpr (sizeof(Rl) == 4) {
                // scale is a power of two: s (Kx - 1) is exact
                const float4 sa{a.x * scale, a.y * scale, a.z * scale, a.w * scale};
                // the row factors by[t + T m]: KD loads in flight, issued in
                // order ahead of their use (volatile loads are not hoisted
                // further, so at most KD factors occupy registers)
                constexpr int KD = PSS_KD;
                float4 ring[KD];
                if constexpr (nls_ky_smem(N)) {
                    // element y = t + T m of the table, folded to min(y, N - y)
                    const unsigned lo = smem_u32(nls_ky_cache<N / 2 + 1>()) + 16u * unsigned(t);
                    const unsigned hi = smem_u32(nls_ky_cache<N / 2 + 1>()) + 16u * unsigned(N - t);
                    auto ky = [&](int m) {
                        return T * m <= N / 2 - T ? lds_f4(lo + 16u * unsigned(T * m))
                                                  : lds_f4(hi - 16u * unsigned(T * m));
                    };
#pragma unroll
                    for (int m = 0; m < KD && m < P; ++m) ring[m] = ky(m);
#pragma unroll
                    for (int m = 0; m < P; ++m) {
                        const float4 b = ring[m % KD];
                        if (m + KD < P) ring[m % KD] = ky(m + KD);
                        v[m] = apply_km1(apply_skm1(v[m], scale, sa), b);
                    }
                } else {
                    const float4 *bp = byl + t;
#pragma unroll
                    for (int m = 0; m < KD && m < P; ++m) ring[m] = ldg_nc_f4(bp + T * m);
#pragma unroll
                    for (int m = 0; m < P; ++m) {
                        const float4 b = ring[m % KD];
                        if (m + KD < P) ring[m % KD] = ldg_nc_f4(bp + T * (m + KD));
                        v[m] = apply_km1(apply_skm1(v[m], scale, sa), b);
                    }
                }
            } else {
#pragma unroll
                for (int m = 0; m < P; ++m) {
                    // scale is a power of two: exact
                    const V2<Rl> z = apply_km1(cscale(v[m], scale), a);
                    v[m] = apply_km1(z, __ldg(byl + t + T * m));
                }
            }
        };
        if constexpr (PSS_SHARED_FFT && sizeof(Rl) == 4) {
#pragma unroll 1
            for (int pass = 0; pass < 2; ++pass) {
                block_fft<N, P, -1, BLOCK>(v, sm, t, tw, [&]() {
                    if (pass == 1) hook();
                });
                if (pass == 0) {
                    propagate();
                    conj_all(v);
                }
            }
            conj_all(v);
        } else {
            block_fft<N, P, -1, BLOCK>(v, sm, t, tw);
            fence(v);
            propagate();
            fence(v);
            block_fft<N, P, +1, BLOCK>(v, sm, t, tw, hook);
        }
        if constexpr (STORE) store_line<P, T>(v, p, nx, t, true);
    }
};

template <class Rl>
cudaError_t nls_row_pass(V2<Rl> *data, int64_t nx, int64_t rows_total, Rl sigma_dt,
                         const TW<Rl> *twx, cudaStream_t s)
{
    return launch_row<Rl>(nx, NlsRow<Rl>{data, sigma_dt}, twx, rows_total, s);
}

template <class Rl>
cudaError_t nls_col_pass(V2<Rl> *data, int64_t nx, int64_t ny, int64_t batch, Rl scale,
                         const TW<Rl> *ax, const TW<Rl> *by, const TW<Rl> *twy, int *status, cudaStream_t s)
{
    return launch_col<Rl>(ny, nx, NlsCol<Rl>{data, nx, scale, ax, by, status}, twy, batch, s);
}

#define PSS_INST(Rl)                                                                            \
    template cudaError_t nls_row_pass<Rl>(V2<Rl> *, int64_t, int64_t, Rl, const TW<Rl> *,        \
                                          cudaStream_t);                                          \
    template cudaError_t nls_col_pass<Rl>(V2<Rl> *, int64_t, int64_t, int64_t, Rl,               \
                                          const TW<Rl> *, const TW<Rl> *, const TW<Rl> *, int *, \
                                          cudaStream_t);
PSS_INST(float)
PSS_INST(double)

}  // namespace pss
