// Stockham FFT building blocks for sm_103a.
//
// A length-N transform is carried by T = N/P threads that each hold P points in
// registers.  Stage s has radix R_s (P, or a smaller power of two for the last
// stage) and span Ns = R_0 ... R_{s-1}; butterfly j (0 <= j < N/R) reads
// elements j + r N/R, multiplies element r by W_{Ns R}^{(j mod Ns) r}, takes an
// R-point DFT in registers and writes output r to (j div Ns) Ns R + (j mod Ns)
// + r Ns (the self-sorting Stockham order).  Thread t owns butterflies
// j = t + q T, so its register m always holds element t + T m: the first stage
// reads, and the last stage writes, unit-stride runs across threads, which is
// what makes the global loads and stores of the row and column passes
// coalesced.  Between stages the points are exchanged through shared memory.
//
// Twiddles W_N^e = exp(-2 pi i e / N) come from a table computed in FP64 on
// the host; the small-radix constants are exact decimal expansions.  In FP32
// every constant is carried as a high and a low part and applied with one
// rounding (cmul_hl), which removes the systematic gain or loss of |z| that
// a rounded constant would repeat in every pass of every step.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "internal.h"

namespace pss {

template <class V> __device__ __forceinline__ V cadd(V a, V b) { return {a.x + b.x, a.y + b.y}; }
template <class V> __device__ __forceinline__ V csub(V a, V b) { return {a.x - b.x, a.y - b.y}; }
// FP32: one packed-pair add per complex add or subtract (each lane rounds as
// a single add does, so the results are those of two adds; the passes are
// bound by instruction issue, and the butterflies are mostly adds: measured
// at 1024^2, row pass 134.8 -> 130.7 us, column pass 155.6 -> 145.5 us)
template <> __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, float2{-b.x, -b.y}); }
template <class V> __device__ __forceinline__ V cmul(V a, V b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <class V> __device__ __forceinline__ V cmulc(V a, V b)
{
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <class V, class R> __device__ __forceinline__ V cscale(V a, R s) { return {a.x * s, a.y * s}; }

// multiply by exp(DIR * i * pi / 2) = DIR * i
template <int DIR, class V> __device__ __forceinline__ V mul_i(V a)
{
    if (DIR > 0) return {-a.y, a.x};
    return {a.y, -a.x};
}

// cos(pi j / 16), j = 0..8
__host__ __device__ constexpr double cos_pi16(int j)
{
    return j == 0 ? 1.0
         : j == 1 ? 0.98078528040323044912618223613424
         : j == 2 ? 0.92387953251128675612818318939679
         : j == 3 ? 0.83146961230254523707878837761791
         : j == 4 ? 0.70710678118654752440084436210485
         : j == 5 ? 0.55557023301960222474283081394853
         : j == 6 ? 0.38268343236508977172845998403040
         : j == 7 ? 0.19509032201612826784828486847702
                  : 0.0;
}
// cos and sin of 2 pi m / 32 for 0 <= m < 16
__host__ __device__ constexpr double cos32(int m) { return m <= 8 ? cos_pi16(m) : -cos_pi16(16 - m); }
__host__ __device__ constexpr double sin32(int m) { return m <= 8 ? cos_pi16(8 - m) : cos_pi16(m - 8); }

// z (hr + lr + i (hi + li)) with one rounding of the exact constant per
// output component: the small product with the low part is folded in inside
// the fused multiply-adds, so the rounding error of the stored high part does
// not bias the result (it would otherwise shrink or grow |z| by the same
// factor in every pass).
__device__ __forceinline__ float2 cmul_hl(float2 z, float hr, float hi, float lr, float li)
{
    const float cr = __fmaf_rn(z.x, lr, -z.y * li);
    const float ci = __fmaf_rn(z.x, li, z.y * lr);
    return {__fmaf_rn(z.x, hr, __fmaf_rn(-z.y, hi, cr)), __fmaf_rn(z.x, hi, __fmaf_rn(z.y, hr, ci))};
}

// twiddle product z * w (forward) or z * conj(w) (inverse)
template <int DIR> __device__ __forceinline__ float2 twmul(float2 z, float4 w)
{
    if (DIR < 0) return cmul_hl(z, w.x, w.y, w.z, w.w);
    return cmul_hl(z, w.x, -w.y, w.z, -w.w);
}
template <int DIR> __device__ __forceinline__ double2 twmul(double2 z, double2 w)
{
    return DIR < 0 ? cmul(z, w) : cmulc(z, w);
}

// s * x with s = hi + lo held exactly to one rounding
__device__ __forceinline__ float mul_hl(float x, float h, float l) { return __fmaf_rn(x, h, x * l); }

// z * exp(DIR * 2 pi i k / RAD), 0 <= k < RAD, RAD | 32
template <int RAD, int DIR, int K, class V> __device__ __forceinline__ V rot(V z)
{
    using R = decltype(z.x);
    constexpr int m = K * (32 / RAD);
    if constexpr (m >= 16) {
        // exp(i (phi + pi)) = -exp(i phi): the negation folds into the adds that follow
        const V r = rot<32, DIR, m - 16>(z);
        return {-r.x, -r.y};
    } else if constexpr (m == 0) {
        return z;
    } else if constexpr (m == 8) {
        return mul_i<DIR>(z);
    } else if constexpr (m == 4 || m == 12) {
        // (c, s) = (sc h, ss h) with h = 1/sqrt(2): c x - s y = h (sc x - ss y)
        constexpr double H = 0.70710678118654752440084436210485;
        constexpr R sc = (m == 4) ? R(1) : R(-1);
        constexpr R ss = DIR > 0 ? R(1) : R(-1);
        const R dr = sc * z.x - ss * z.y, di = sc * z.y + ss * z.x;
        if constexpr (sizeof(R) == 4) {
            constexpr float hh = float(H), hl = float(H - double(float(H)));
            // both components at once as packed pairs (each lane rounds as
            // mul_hl does; measured about 1 % off both NLS passes at 1024^2;
            // the general rotations below stay scalar: their operand pairs
            // would need swapped copies, and a packed form was 9 % slower)
            const float2 d{dr, di};
            return __ffma2_rn(d, float2{hh, hh}, __fmul2_rn(d, float2{hl, hl}));
        } else {
            return {R(H) * dr, R(H) * di};
        }
    } else {
        constexpr double c = cos32(m), s = DIR > 0 ? sin32(m) : -sin32(m);
        if constexpr (sizeof(R) == 4) {
            constexpr float ch = float(c), sh = float(s);
            constexpr float cl = float(c - double(ch)), sl = float(s - double(sh));
            return cmul_hl(z, ch, sh, cl, sl);
        } else {
            return {R(c) * z.x - R(s) * z.y, R(c) * z.y + R(s) * z.x};
        }
    }
}

// One split-radix step (decimation in frequency) of the RAD-point DFT of
// v[0], v[S], ..., v[(RAD-1) S], for k = K .. RAD/4 - 1 (a, b, c, d =
// elements k, k + RAD/4, k + RAD/2, k + 3 RAD/4; w = exp(DIR 2 pi i / RAD)):
// the even outputs are the RAD/2-point DFT of (a + c, b + d), outputs 4j + 1
// the RAD/4-point DFT of (a - c + DIR i (b - d)) w^k and outputs 4j + 3 that
// of (a - c - DIR i (b - d)) w^{3k}.  Against plain radix-2 steps this needs
// fewer non-trivial rotations (16 instead of 20 general ones and 10 instead
// of 14 by odd multiples of pi/4 for 32 points), with the same additions.
template <int RAD, int DIR, int S, int K, class V> __device__ __forceinline__ void sr_level(V *v)
{
    if constexpr (K < RAD / 4) {
        constexpr int Q = RAD / 4;
        const V a = v[K * S], b = v[(K + Q) * S], c = v[(K + 2 * Q) * S], d = v[(K + 3 * Q) * S];
        v[K * S] = cadd(a, c);
        v[(K + Q) * S] = cadd(b, d);
        const V t1 = csub(a, c), jt2 = mul_i<DIR>(csub(b, d));
        v[(K + 2 * Q) * S] = rot<RAD, DIR, K>(cadd(t1, jt2));
        v[(K + 3 * Q) * S] = rot<RAD, DIR, 3 * K>(csub(t1, jt2));
        sr_level<RAD, DIR, S, K + 1>(v);
    }
}

// In-register DFT of RAD points v[0], v[S], ..., v[(RAD-1) S] by split-radix
// decimation in frequency; the result is left in bit-reversed order (output
// r at position bitrev(r)): the even outputs fill the first half, outputs
// 4j + 1 the third quarter and 4j + 3 the last.
template <int RAD, int DIR, int S, class V> __device__ __forceinline__ void dft_dif(V *v)
{
    if constexpr (RAD == 2) {
        const V a = v[0], b = v[S];
        v[0] = cadd(a, b);
        v[S] = csub(a, b);
    } else if constexpr (RAD >= 4) {
        sr_level<RAD, DIR, S, 0>(v);
        dft_dif<RAD / 2, DIR, S>(v);
        dft_dif<RAD / 4, DIR, S>(v + (RAD / 2) * S);
        dft_dif<RAD / 4, DIR, S>(v + (3 * RAD / 4) * S);
    }
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
// bit reversal of the low `bits` bits of r; a loop (not recursion) so that it
// folds to a constant inside unrolled loops and register arrays stay in
// registers
__host__ __device__ __forceinline__ constexpr int bitrev(int r, int bits)
{
    int o = 0;
    for (int i = 0; i < bits; ++i) o = (o << 1) | ((r >> i) & 1);
    return o;
}

// Stage list of a length-N transform with P points per thread.
template <int N, int P> struct Plan {
    static_assert((N & (N - 1)) == 0 && (P & (P - 1)) == 0 && P <= N && P <= 32, "bad plan");
    static constexpr int T = N / P;
    static constexpr int LOGN = ilog2(N), LOGP = ilog2(P);
    static constexpr int FULL = LOGN / LOGP, REM = LOGN % LOGP;
    static constexpr int STAGES = FULL + (REM ? 1 : 0);
    __host__ __device__ static constexpr int radix(int s) { return s < FULL ? P : (1 << REM); }
    __host__ __device__ static constexpr int span(int s) { return s == 0 ? 1 : span(s - 1) * radix(s - 1); }
};

// Shared-memory view of one transform's N points with one pad slot every
// 2^PADLOG points (breaks the power-of-two strides of the Stockham writes).
template <class V, int PADLOG> struct SmemLine {
    V *base;
    __host__ __device__ static constexpr int padded(int n) { return n + (n >> PADLOG); }
    __device__ __forceinline__ V &operator[](int i) const { return base[i + (i >> PADLOG)]; }
};

// The twiddle loads of a stage do not depend on the data, so the compiler
// would issue those of every stage of every transform in a kernel up front
// and hold them all in registers (hundreds for the two transforms of a fused
// pass).  Passing the table pointer through a volatile move after the
// stage's exchange barrier keeps each stage's loads after that barrier.
template <class W> __device__ __forceinline__ const W *launder(const W *p)
{
    const W *q;
    asm volatile("mov.b64 %0, %1;" : "=l"(q) : "l"(p));
    return q;
}

// Ask for the line holding p to be brought into L2 (no register is written):
// used at the start of a tile for the arrays its update reads later, so those
// loads wait for L2 rather than for HBM.
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Load of streamed state (read once per pass, or re-read from L2 right after
// this thread stored it): cached in L2 only, so that it does not evict the
// small tables (wavenumbers, masks, twiddles) the pass keeps reading through
// L1.  PSS_LDCG=0 uses ordinary loads.
#ifndef PSS_LDCG
#define PSS_LDCG 1
#endif
template <class V> __device__ __forceinline__ V ld_stream(const V *p)
{
#if PSS_LDCG
    return __ldcg(p);
#else
    return *p;
#endif
}

// Register fence: every value of v is materialised here and nothing that
// uses v moves above it, so the two transforms of a fused pass are not
// interleaved (which would keep both transforms' temporaries live).
template <int P> __device__ __forceinline__ void fence(float2 (&v)[P])
{
#pragma unroll
    for (int m = 0; m < P; ++m) asm volatile("" : "+f"(v[m].x), "+f"(v[m].y));
}
template <int P> __device__ __forceinline__ void fence(double2 (&v)[P])
{
#pragma unroll
    for (int m = 0; m < P; ++m) asm volatile("" : "+d"(v[m].x), "+d"(v[m].y));
}

// One copy of the forward transform can serve both transforms of a fused
// pass: F^-1 x = conj(F conj x) exactly (negation is exact), which halves the
// unrolled code and the registers it holds.
template <int P, class V> __device__ __forceinline__ void conj_all(V (&v)[P])
{
#pragma unroll
    for (int m = 0; m < P; ++m) v[m].y = -v[m].y;
}

// Barrier among the threads that share a transform's shared-memory line.
// SYNC = 0: the transform lives within one warp; SYNC = 1: it spans the
// CTA; SYNC = G > 1 (a multiple of 32): the CTA holds several transforms of
// G consecutive threads each (rows of a row pass), and each group waits only
// for itself, on named barrier 1 + threadIdx.x / G.
template <int SYNC> __device__ __forceinline__ void fft_sync()
{
    if constexpr (SYNC == 0) {
        __syncwarp();
    } else if constexpr (SYNC == 1) {
        __syncthreads();
    } else {
        static_assert(SYNC % 32 == 0, "whole warps per group");
        asm volatile("bar.sync %0, %1;" ::"r"(1 + int(threadIdx.x) / SYNC), "n"(SYNC) : "memory");
    }
}

// A transform's caller may pass a hook that runs once, at the start of the
// last stage: by then this thread has made its last shared-memory access of
// the transform, so a pass can start refilling the buffer for its next tile
// while the last stage computes.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// FP32 transforms read the twiddles of their second stage (span NS = P,
// radix R: NS (R - 1) values W_{NS R}^{jm r}) from a copy in shared memory
// laid out [r - 1][jm], so that the threads of a warp, whose jm are
// consecutive (or equal), read consecutive 16-byte words: no bank conflicts,
// and shared-memory latency instead of a global load's.  Every kernel that
// runs a FP32 transform of length N fills the copy once (fill_stage_tw) and
// synchronises before its first transform.  PSS_SMEM_TW=0 reads every stage
// from the global table instead.
#ifndef PSS_SMEM_TW
#define PSS_SMEM_TW 1
#endif
// twiddle loads of the shared copy kept in flight per thread
#ifndef PSS_TWD
#define PSS_TWD 4
#endif
template <int N, int P> struct StageTw {
    using PL = Plan<N, P>;
    static constexpr bool ON = PSS_SMEM_TW && PL::STAGES >= 2;
    static constexpr int NS = ON ? PL::span(1) : 1, R = ON ? PL::radix(1) : 2;
    static constexpr int COUNT = NS * (R - 1);
};
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// a 16-byte shared-memory load kept in program order
__device__ __forceinline__ float4 lds_f4(unsigned addr)
{
    float4 r;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "r"(addr));
    return r;
}
// the copy of one (span, radix): a static shared array of the kernel
template <int NS, int R> __device__ __forceinline__ float4 *stage_tw_smem()
{
    __shared__ __align__(16) float4 cache[NS * (R - 1)];
    return cache;
}
// all threads of the CTA: copy the second stage's twiddles of a length-N
// transform from the global table; the caller synchronises afterwards
template <int N, int P> __device__ __forceinline__ void fill_stage_tw(const float4 *__restrict__ tw)
{
    using ST = StageTw<N, P>;
    if constexpr (ST::ON) {
        float4 *c = stage_tw_smem<ST::NS, ST::R>();
        for (int e = int(threadIdx.x); e < ST::COUNT; e += int(blockDim.x)) {
            const int r = e / ST::NS + 1, jm = e % ST::NS;
            c[e] = __ldg(tw + jm * r * (N / (ST::NS * ST::R)));
        }
    }
}
template <int N, int P> __device__ __forceinline__ void fill_stage_tw(const double2 *) {}

// Last-stage twiddles of FP32 transforms with several butterflies per thread
// (Q > 1: three or more stages) as W_N^{t r} (loaded) times W_P^{q r} (a
// compile-time rotation): R - 1 table loads per thread instead of Q (R - 1),
// and a 16-byte-per-thread footprint of the table instead of the whole last
// stage's.  Each factor is applied with one rounding of its exact hi + lo
// value.  PSS_TW_FACTOR=0 loads every product from the table.
#ifndef PSS_TW_FACTOR
#define PSS_TW_FACTOR 1
#endif
template <int P, int DIR, int Q, int RR, int q, class V, class W>
__device__ __forceinline__ void fact_rot(V *v, const W &w)
{
    if constexpr (q < Q) {
        v[q + RR * Q] = rot<P, DIR, (q * RR) % P>(twmul<DIR>(v[q + RR * Q], w));
        fact_rot<P, DIR, Q, RR, q + 1>(v, w);
    }
}
template <int P, int DIR, int Q, int R, int RR, class V, class W>
__device__ __forceinline__ void fact_stage(V *v, const W *__restrict__ tw, int t)
{
    if constexpr (RR < R) {
        const W w = __ldg(tw + t * RR);
        fact_rot<P, DIR, Q, RR, 0>(v, w);
        fact_stage<P, DIR, Q, R, RR + 1>(v, tw, t);
    }
}

// One Stockham stage s of a length-N transform (DIR = -1 forward, +1 inverse).
// On entry register m holds element t + T m of the stage input; on exit (for
// the last stage) register m holds output element t + T m.  Other stages leave
// their output in shared memory and reload the next stage's input.
template <int N, int P, int DIR, int S, int BLOCK, class V, class Sm, class W, class H>
__device__ __forceinline__ void fft_stage(V (&v)[P], const Sm &sm, int t, const W *__restrict__ tw, const H &hook)
{
    using PL = Plan<N, P>;
    constexpr int R = PL::radix(S), NS = PL::span(S), T = PL::T, Q = P / R;
    constexpr bool LAST = (S == PL::STAGES - 1);
    if constexpr (LAST) hook();
    if constexpr (S > 0) {
        // twiddles W_{NS R}^{(j mod NS) r} = W_N^{(j mod NS) r N/(NS R)}
        constexpr bool SMEM = S == 1 && std::is_same<W, float4>::value && StageTw<N, P>::ON;
        constexpr bool FACT = PSS_TW_FACTOR && LAST && !SMEM && Q > 1 && std::is_same<W, float4>::value;
        static_assert(!FACT || NS == T * Q, "last stage: jm = t + T q");
        tw = launder(tw);
#pragma unroll
        for (int q = 0; q < (FACT ? 0 : Q); ++q) {
            const int jm = (t + q * T) & (NS - 1);
            if constexpr (SMEM) {
                static_assert(NS == StageTw<N, P>::NS && R == StageTw<N, P>::R, "stage 1 shape");
                // TWD loads in flight, issued in order (volatile loads are not
                // hoisted further, so at most TWD twiddles occupy registers)
                constexpr int TWD = PSS_TWD;
                const unsigned a0 = smem_u32(stage_tw_smem<NS, R>()) + unsigned(jm) * 16u;
                float4 ring[TWD];
#pragma unroll
                for (int r = 1; r < R && r <= TWD; ++r) ring[r - 1] = lds_f4(a0 + unsigned((r - 1) * NS) * 16u);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const float4 w = ring[(r - 1) % TWD];
                    if (r + TWD < R) ring[(r - 1) % TWD] = lds_f4(a0 + unsigned((r + TWD - 1) * NS) * 16u);
                    v[q + r * Q] = twmul<DIR>(v[q + r * Q], w);
                }
            } else if constexpr (!FACT) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const W w = __ldg(tw + jm * r * (N / (NS * R)));
                    v[q + r * Q] = twmul<DIR>(v[q + r * Q], w);
                }
            }
        }
        // the last stage (span NS = N / R = T Q): jm = t + T q, so
        // W_N^{jm r} = W_N^{t r} W_P^{q r}: R - 1 loads per thread and a
        // constant rotation per butterfly
        if constexpr (FACT) fact_stage<P, DIR, Q, R, 1>(v, tw, t);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) dft_dif<R, DIR, Q>(v + q);
    constexpr int BITS = ilog2(R);
    if constexpr (LAST) {
        // undo the bit reversal: output r of butterfly q sits in v[q + bitrev(r) Q]
        V o[P];
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int r = 0; r < R; ++r) o[q + r * Q] = v[q + bitrev(r, BITS) * Q];
#pragma unroll
        for (int m = 0; m < P; ++m) v[m] = o[m];
    } else {
        fft_sync<BLOCK>();  // previous readers of shared memory are done
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int j = t + q * T;
            const int base = (j / NS) * NS * R + (j & (NS - 1));
#pragma unroll
            for (int r = 0; r < R; ++r) sm[base + r * NS] = v[q + bitrev(r, BITS) * Q];
        }
        fft_sync<BLOCK>();
#pragma unroll
        for (int m = 0; m < P; ++m) v[m] = sm[t + T * m];
    }
}

template <int N, int P, int DIR, int S, int BLOCK, class V, class Sm, class W, class H>
__device__ __forceinline__ void fft_stages(V (&v)[P], const Sm &sm, int t, const W *__restrict__ tw, const H &hook)
{
    if constexpr (S < Plan<N, P>::STAGES) {
        fft_stage<N, P, DIR, S, BLOCK>(v, sm, t, tw, hook);
        fft_stages<N, P, DIR, S + 1, BLOCK>(v, sm, t, tw, hook);
    }
}

// Full unnormalised length-N transform of the points held by the T threads
// t = 0..T-1 (register m = element t + T m, in and out).
template <int N, int P, int DIR, int BLOCK, class V, class Sm, class W, class H = NoHook>
__device__ __forceinline__ void block_fft(V (&v)[P], const Sm &sm, int t, const W *__restrict__ tw,
                                          const H &hook = H{})
{
    fft_stages<N, P, DIR, 0, BLOCK>(v, sm, t, tw, hook);
}

}  // namespace pss
