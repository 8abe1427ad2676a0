// Row and column pass kernels.
//
// A row pass transforms along x (contiguous rows of length NX); a CTA holds
// ROWS rows, each carried by T = NX/P threads.  A column pass transforms along
// y; a CTA holds W adjacent columns of length NY, thread (c, t) with the column
// index c fastest so that a warp's loads cover 32/W rows of W contiguous
// points.  The equation-specific work is an "op" that loads its inputs, calls
// block_fft around its pointwise or k-space arithmetic and stores its outputs,
// so each pass is exactly one read and one write of every array it touches.
#pragma once
#include "fft_core.cuh"

namespace pss {

// ----------------------------------------------------------------------------
// Per (precision, length) launch shapes.
template <class Rl> struct Shape {
    static constexpr int ESZ = 2 * int(sizeof(Rl));
    // points per thread of the row and column transforms
    __host__ __device__ static constexpr int rowP(int n) { return n < 16 ? n : 16; }
    __host__ __device__ static constexpr int colP(int n) { return n < 16 ? n : 16; }
    // rows per CTA: about 256 threads
    __host__ __device__ static constexpr int rows(int n)
    {
        return (n / rowP(n)) >= 256 ? 1 : 256 / (n / rowP(n));
    }
    // columns per CTA: 64-byte row segments when shared memory and the
    // register budget (512 threads FP32, 256 FP64) allow
    __host__ __device__ static constexpr int cols(int n)
    {
        int w = sizeof(Rl) == 4 ? 8 : 4;
        const int tmax = sizeof(Rl) == 4 ? 512 : 256;
        while (w > 1 && ((long)w * (n + n / 16) * ESZ > 150 * 1024 || w * (n / colP(n)) > tmax)) w /= 2;
        return w;
    }
};

// shared-memory pad period of a transform with P points per thread
__host__ __device__ constexpr int pad_log(int P) { return P < 2 ? 30 : ilog2(P); }

// Max number of distinct 4-byte words any bank serves when a warp of W-wide
// column groups touches element c*S + dt (c < W, dt < 32/W) of ESZ bytes each.
__host__ __device__ constexpr int bank_load(int S, int W, int ESZ)
{
    int cnt[32] = {};
    int mx = 0;
    const int tper = 32 / W;
    for (int c = 0; c < W; ++c)
        for (int dt = 0; dt < tper; ++dt)
            for (int w = 0; w < ESZ / 4; ++w) {
                const int b = ((c * S + dt) * (ESZ / 4) + w) & 31;
                if (++cnt[b] > mx) mx = cnt[b];
            }
    return mx;
}
// column stride (in elements) >= base with the least bank load
__host__ __device__ constexpr int col_stride(int base, int W, int ESZ)
{
    int best = base;
    for (int d = 1; d < 32; ++d)
        if (bank_load(base + d, W, ESZ) < bank_load(best, W, ESZ)) best = base + d;
    return best;
}

template <class Rl, int N> struct RowCfg {
    static constexpr int P = Shape<Rl>::rowP(N), T = N / P, ROWS = Shape<Rl>::rows(N);
    static constexpr int PADLOG = pad_log(P);
    static constexpr int LINE = N + (N >> PADLOG);
    static constexpr int THREADS = ROWS * T;
    static constexpr bool BLOCK = T > 32;
    static constexpr size_t SMEM = (T > 1) ? size_t(ROWS) * LINE * Shape<Rl>::ESZ : 0;
};

template <class Rl, int N> struct ColCfg {
    static constexpr int P = Shape<Rl>::colP(N), T = N / P, W = Shape<Rl>::cols(N);
    static constexpr int PADLOG = pad_log(P);
    static constexpr int STRIDE = col_stride(N + (N >> PADLOG), W, Shape<Rl>::ESZ);
    static constexpr int THREADS = W * T;
    static constexpr bool BLOCK = THREADS > 32;
    static constexpr size_t SMEM = (T > 1) ? size_t(W) * STRIDE * Shape<Rl>::ESZ : 0;
};

// ----------------------------------------------------------------------------
// Kernel shells

// rows_total = batch * ny; row r of the batch starts at element r * NX
template <class Rl, int N, class Op>
__global__ void __launch_bounds__(RowCfg<Rl, N>::THREADS)
    k_row(Op op, const TW<Rl> *__restrict__ tw, int64_t rows_total)
{
    using C = RowCfg<Rl, N>;
    using V = V2<Rl>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lr = threadIdx.x / C::T, t = threadIdx.x % C::T;
    SmemLine<V, C::PADLOG> sm{reinterpret_cast<V *>(smem_raw) + lr * C::LINE};
    const int64_t row = int64_t(blockIdx.x) * C::ROWS + lr;
    op.template run<N, C::P, C::BLOCK>(row, row < rows_total, t, sm, tw);
}

// grid (NX / W, batch); column x of field b
template <class Rl, int N, class Op>
__global__ void __launch_bounds__(ColCfg<Rl, N>::THREADS)
    k_col(Op op, const TW<Rl> *__restrict__ tw)
{
    using C = ColCfg<Rl, N>;
    using V = V2<Rl>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = threadIdx.x % C::W, t = threadIdx.x / C::W;
    SmemLine<V, C::PADLOG> sm{reinterpret_cast<V *>(smem_raw) + c * C::STRIDE};
    op.template run<N, C::P, C::BLOCK>(int64_t(blockIdx.y), int(blockIdx.x) * C::W + c, t, sm, tw);
}

// ----------------------------------------------------------------------------
// Load/store helpers: register m <-> element t + T m of a line with stride ST
template <int P, int T, class V>
__device__ __forceinline__ void load_line(V (&v)[P], const V *__restrict__ p, int64_t st, int t,
                                          bool ok)
{
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = ok ? p[int64_t(t + T * m) * st] : V{0, 0};
}
template <int P, int T, class V>
__device__ __forceinline__ void store_line(const V (&v)[P], V *__restrict__ p, int64_t st, int t,
                                           bool ok)
{
    if (!ok) return;
#pragma unroll
    for (int m = 0; m < P; ++m) p[int64_t(t + T * m) * st] = v[m];
}

// ----------------------------------------------------------------------------
// Plain transforms (the 2D FFT of every step, Section 4)

template <class Rl, int DIR> struct RowFft {
    V2<Rl> *data;
    Rl scale;  // applied after the transform when != 1
    template <int N, int P, bool BLOCK, class Sm>
    __device__ __forceinline__ void run(int64_t row, bool ok, int t, const Sm &sm,
                                        const TW<Rl> *tw) const
    {
        constexpr int T = N / P;
        V2<Rl> v[P];
        V2<Rl> *p = data + row * N;
        load_line<P, T>(v, p, 1, t, ok);
        block_fft<N, P, DIR, BLOCK>(v, sm, t, tw);
        if (scale != Rl(1))
#pragma unroll
            for (int m = 0; m < P; ++m) v[m] = cscale(v[m], scale);
        store_line<P, T>(v, p, 1, t, ok);
    }
};

template <class Rl, int DIR> struct ColFft {
    V2<Rl> *data;
    int64_t nx;
    Rl scale;
    template <int N, int P, bool BLOCK, class Sm>
    __device__ __forceinline__ void run(int64_t field, int x, int t, const Sm &sm,
                                        const TW<Rl> *tw) const
    {
        constexpr int T = N / P;
        V2<Rl> v[P];
        V2<Rl> *p = data + field * N * nx + x;
        load_line<P, T>(v, p, nx, t, true);
        block_fft<N, P, DIR, BLOCK>(v, sm, t, tw);
        if (scale != Rl(1))
#pragma unroll
            for (int m = 0; m < P; ++m) v[m] = cscale(v[m], scale);
        store_line<P, T>(v, p, nx, t, true);
    }
};

}  // namespace pss
