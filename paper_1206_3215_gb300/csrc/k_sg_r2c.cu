// Sine-Gordon step (Eq. 3, Section 4.2) on half spectra: u is real, so its
// Fourier coefficients for kx < 0 are the complex conjugates of those for
// kx > 0 and only kx = 0 .. N/2 are kept (the paper's own programs use
// real-to-complex transforms for this equation, Section 5.2).  Both passes
// then move about half the bytes of the complex-to-complex step.
//
// Layout: complex [batch][ny][sx], sx >= N/2 + 1; columns 0 .. N/2 hold the
// half spectrum in x, the columns beyond hold zeros (the column pass carries
// them along unchanged).
//
// The row pass turns H (x: half spectrum, y: physical) into S, the half
// spectrum in x of sin u.  A row of N real points u_n is handled as M = N/2
// complex points z_j = u_{2j} + i u_{2j+1}.  From the half spectrum X_0 .. X_M
// of u (and X_{M+k} = conj X_{M-k}):
//   Z_k = (X_k + conj X_{M-k}) + i e^{2 pi i k/N} (X_k - conj X_{M-k}),  k < M,
//   z = unnormalised inverse DFT_M of Z.
// After s = sin u, the forward DFT_M W of w_j = s_{2j} + i s_{2j+1} gives
//   A_k = (W_k + conj W_{M-k}) / 2,   B_k = -i (W_k - conj W_{M-k}) / 2,
//   S_k = A_k + e^{-2 pi i k/N} B_k  (k < M),   S_M = A_0 - B_0,
// where A and B are the DFTs of the even and odd samples of s.  The column
// pass is the complex one of k_sg.cu applied to the sx columns.
#include "launch.cuh"
#include "sg_sin.cuh"

namespace pss {

namespace {

template <class Rl, int M> struct R2cCfg {
    static constexpr int P = Shape<Rl>::rowP(M);
    static constexpr int T = M / P;
    static constexpr int ROWS = T >= 256 ? 1 : 256 / T;
    static constexpr int THREADS = ROWS * T;
    // barrier of one row's threads (fft_sync): a warp (T <= 32: the rows are
    // warp-local), the CTA, or the row's own named barrier
    static constexpr int BLOCK = T <= 32 ? 0 : (ROWS > 1 ? T : 1);
    static constexpr int PADLOG = pad_log(P);
    static constexpr int LINE = M + (M >> PADLOG) + 2;  // the padded line plus X_M
    static constexpr size_t SMEM = size_t(ROWS) * LINE * sizeof(V2<Rl>);
    static constexpr int MIN_CTAS = (sizeof(Rl) == 4 && THREADS * 2 <= 512) ? 2 : 1;
};

// rows_total = batch * ny rows of stride sx; twm: length-M transform
// twiddles, twn: length-N twiddles (e^{-2 pi i e / N}, e < N)
template <class Rl, int M>
__global__ void __launch_bounds__(R2cCfg<Rl, M>::THREADS, R2cCfg<Rl, M>::MIN_CTAS)
    k_sg_row_r2c(V2<Rl> *__restrict__ h, int64_t sx, int64_t rows_total, const TW<Rl> *__restrict__ twm,
                 const TW<Rl> *__restrict__ twn)
{
    using C = R2cCfg<Rl, M>;
    using V = V2<Rl>;
    using Sm = SmemLine<V, C::PADLOG>;
    constexpr int P = C::P, T = C::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int rl = threadIdx.x / T, t = threadIdx.x % T;
    const Sm sm{reinterpret_cast<V *>(smem_raw) + rl * C::LINE};
    fill_stage_tw<M, P>(twm);
    __syncthreads();
    for (int64_t r0 = int64_t(blockIdx.x) * C::ROWS; r0 < rows_total; r0 += int64_t(gridDim.x) * C::ROWS) {
        const int64_t row = r0 + rl;
        const bool ok = row < rows_total;
        V *const p = h + (ok ? row : int64_t(0)) * sx;
        // stage X_0 .. X_M of the row (every thread reads two of them below)
        fft_sync<C::BLOCK>();  // the previous row's last readers are done
        if (ok) {
#pragma unroll
            for (int m = 0; m < P; ++m) cp_async<sizeof(V)>(&sm[t + T * m], p + t + T * m);
            if (t == 0) cp_async<sizeof(V)>(&sm[M], p + M);
        }
        cp_async_commit();
        cp_async_wait<0>();
        fft_sync<C::BLOCK>();
        V v[P];
        const TW<Rl> *tn = launder(twn);
#pragma unroll
        for (int m = 0; m < P; ++m) {
            const int k = t + T * m;
            const V x = sm[k], xp = sm[M - k];
            const V e{x.x + xp.x, x.y - xp.y};                           // X_k + conj X_{M-k}
            const V o = twmul<+1>(V{x.x - xp.x, x.y + xp.y}, __ldg(tn + k));  // e^{2 pi i k/N} (X_k - conj X_{M-k})
            // conj Z_k: the inverse transform runs as conj(F conj Z)
            v[m] = V{e.x - o.y, -(e.y + o.x)};
        }
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            block_fft<M, P, -1, C::BLOCK>(v, sm, t, twm);
            if (pass == 0)  // z = conj(F conj Z): u_{2j} = Re z, u_{2j+1} = Im z = -Im(F conj Z)
#pragma unroll
                for (int m = 0; m < P; ++m) v[m] = V{sg_sin(v[m].x), sg_sin(-v[m].y)};
        }
        // W_k in registers (k = t + T m); the partner W_{M-k} through shared memory
        fft_sync<C::BLOCK>();
#pragma unroll
        for (int m = 0; m < P; ++m) sm[t + T * m] = v[m];
        fft_sync<C::BLOCK>();
        tn = launder(twn);
        const Rl half = Rl(0.5);
#pragma unroll
        for (int m = 0; m < P; ++m) {
            const int k = t + T * m;
            const V w = v[m], wp = sm[(M - k) & (M - 1)];
            const V a{half * (w.x + wp.x), half * (w.y - wp.y)};  // (W_k + conj W_{M-k}) / 2
            const V b{half * (w.y + wp.y), half * (wp.x - w.x)};  // -i (W_k - conj W_{M-k}) / 2
            const V tb = twmul<-1>(b, __ldg(tn + k));
            if (ok) p[k] = V{a.x + tb.x, a.y + tb.y};
            if (ok && k == 0) p[M] = V{a.x - b.x, a.y - b.y};
        }
    }
    cp_async_wait<0>();
}

template <class Rl, int M>
cudaError_t launch_r2c(V2<Rl> *h, int64_t sx, int64_t rows_total, const TW<Rl> *twm, const TW<Rl> *twn,
                       cudaStream_t s)
{
    using C = R2cCfg<Rl, M>;
    auto k = k_sg_row_r2c<Rl, M>;
    static std::atomic<unsigned> done{0};
    static int ctas[32] = {};
    cudaError_t e = allow_smem(k, C::SMEM, done);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (rows_total + C::ROWS - 1) / C::ROWS;
    if (tiles <= 0) return cudaSuccess;
    int grid = 0;
    if ((e = resident_ctas(k, C::THREADS, C::SMEM, ctas, &grid)) != cudaSuccess) return e;
    if (tiles < grid) grid = int(tiles);
    k<<<dim3(unsigned(grid)), C::THREADS, C::SMEM, s>>>(h, sx, rows_total, twm, twn);
    return cudaGetLastError();
}

// half spectrum <-> full spectrum of real fields ([ny][n] <-> [ny][sx])
template <class Rl>
__global__ void k_pack_half(const V2<Rl> *__restrict__ full, V2<Rl> *__restrict__ half, int64_t n, int64_t ny,
                            int64_t sx, int64_t total)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t x = i % sx, r = i / sx;  // r = field * ny + y
        half[i] = x <= n / 2 ? full[r * n + x] : V2<Rl>{Rl(0), Rl(0)};
    }
}

// full(y, x) = half(y, x) for x <= n/2, conj half(-y mod ny, n - x) otherwise
template <class Rl>
__global__ void k_unpack_half(const V2<Rl> *__restrict__ half, V2<Rl> *__restrict__ full, int64_t n, int64_t ny,
                              int64_t sx, int64_t total)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t x = i % n, r = i / n, y = r % ny, f = r / ny;
        if (x <= n / 2) {
            full[i] = half[r * sx + x];
        } else {
            const V2<Rl> c = half[(f * ny + (ny - y) % ny) * sx + (n - x)];
            full[i] = V2<Rl>{c.x, -c.y};
        }
    }
}

}  // namespace

template <class Rl>
cudaError_t sg_row_pass_r2c(V2<Rl> *h, int64_t nx, int64_t sx, int64_t rows_total, const TW<Rl> *twm,
                            const TW<Rl> *twn, cudaStream_t s)
{
    switch (nx / 2) {
#define PSS_CASE(N) \
    case N: return launch_r2c<Rl, N>(h, sx, rows_total, twm, twn, s);
        PSS_CASE(8) PSS_CASE(16) PSS_CASE(32) PSS_CASE(64) PSS_CASE(128) PSS_CASE(256) PSS_CASE(512)
        PSS_CASE(1024) PSS_CASE(2048) PSS_CASE(4096)
#undef PSS_CASE
    default: return cudaErrorInvalidValue;
    }
}

template <class Rl>
cudaError_t pack_half(const V2<Rl> *full, V2<Rl> *half, int64_t nx, int64_t ny, int64_t sx, int64_t batch,
                      cudaStream_t s)
{
    const int64_t total = sx * ny * batch;
    const unsigned blocks = unsigned(std::min<int64_t>((total + 255) / 256, 4096));
    k_pack_half<Rl><<<blocks, 256, 0, s>>>(full, half, nx, ny, sx, total);
    return cudaGetLastError();
}

template <class Rl>
cudaError_t unpack_half(const V2<Rl> *half, V2<Rl> *full, int64_t nx, int64_t ny, int64_t sx, int64_t batch,
                        cudaStream_t s)
{
    const int64_t total = nx * ny * batch;
    const unsigned blocks = unsigned(std::min<int64_t>((total + 255) / 256, 4096));
    k_unpack_half<Rl><<<blocks, 256, 0, s>>>(half, full, nx, ny, sx, total);
    return cudaGetLastError();
}

#define PSS_INST(Rl)                                                                                        \
    template cudaError_t sg_row_pass_r2c<Rl>(V2<Rl> *, int64_t, int64_t, int64_t, const TW<Rl> *,          \
                                             const TW<Rl> *, cudaStream_t);                                 \
    template cudaError_t pack_half<Rl>(const V2<Rl> *, V2<Rl> *, int64_t, int64_t, int64_t, int64_t,        \
                                       cudaStream_t);                                                       \
    template cudaError_t unpack_half<Rl>(const V2<Rl> *, V2<Rl> *, int64_t, int64_t, int64_t, int64_t,      \
                                         cudaStream_t);
PSS_INST(float)
PSS_INST(double)

}  // namespace pss
