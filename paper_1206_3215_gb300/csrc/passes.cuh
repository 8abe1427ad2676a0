// Row and column pass kernels.
//
// A row pass transforms along x (contiguous rows of length NX); a tile is
// ROWS rows, each carried by T = NX/P threads.  A column pass transforms
// along y; a tile is W adjacent columns of one field, thread (c, t) with the
// column index c fastest so that a warp's accesses cover 32/W rows of W
// contiguous points.
//
// Both are persistent: each CTA walks tiles blockIdx.x, +gridDim.x, ...  With
// two shared-memory buffers, cp.async copies of the next tile's input lines
// are in flight into one while the CTA transforms the tile in the other, so
// HBM stays busy during the arithmetic without holding the data in
// registers.  Each thread copies exactly the points it reads back for the
// first Stockham stage (element t + T m of its line), so it only waits for
// its own copies; the buffer then serves as the exchange space of that
// tile's transforms.  The lean FP32 shape has one buffer per CTA and two
// CTAs per SM: its row passes start the next tile's copies once the last
// transform has made its last shared-memory access, and its column passes
// take each tile by one tensor copy (k_col_tma, below).
//
// The equation-specific work is an "op": it names its staged input arrays
// and, given the staged points in registers, does the transforms around its
// pointwise or k-space arithmetic and stores its outputs, so each pass is
// one read and one write of every array it touches.
#pragma once
#include "fft_core.cuh"
#include "tma.cuh"

#include <type_traits>
#include <utility>

namespace pss {

// ----------------------------------------------------------------------------
// Per (precision, length) launch shapes.  The PSS_* macros let a build pick
// other shapes (points per thread, threads per CTA, resident CTAs per SM).
// Measured at 1024^2 on GB300: 32 points per thread (two radix-32 stages, one
// exchange) is 18% faster than 16 in FP32; FP64 prefers 16.
#ifndef PSS_ROW_P
#define PSS_ROW_P 32
#endif
#ifndef PSS_COL_P
#define PSS_COL_P 32
#endif
#ifndef PSS_BIG_N
#define PSS_BIG_N 2048
#endif
#ifndef PSS_ROW_P_BIG
#define PSS_ROW_P_BIG PSS_ROW_P
#endif
#ifndef PSS_COL_P_BIG
#define PSS_COL_P_BIG PSS_COL_P
#endif
#ifndef PSS_ROW_P64
#define PSS_ROW_P64 16
#endif
#ifndef PSS_COL_P64
#define PSS_COL_P64 16
#endif
#ifndef PSS_ROW_THREADS
#define PSS_ROW_THREADS 256
#endif
#ifndef PSS_COL_THREADS
#define PSS_COL_THREADS 256
#endif
#ifndef PSS_ROW_THREADS_SMALL
#define PSS_ROW_THREADS_SMALL 64
#endif
#ifndef PSS_COL_WIDE_THREADS
#define PSS_COL_WIDE_THREADS 512
#endif
#ifndef PSS_COL_WMAX
#define PSS_COL_WMAX 8
#endif
// FP32 (measured, 1024^2): one shared-memory buffer per CTA and two CTAs per
// SM (<= 128 registers) beat a double-buffered CTA alone by 9 %; FP64 keeps
// the double buffer and one CTA per SM.
#ifndef PSS_MIN_CTAS
#define PSS_MIN_CTAS 2
#endif
#ifndef PSS_MAX_NBUF
#define PSS_MAX_NBUF 1
#endif
#ifndef PSS_THREADS_PER_SM
#define PSS_THREADS_PER_SM 512
#endif
#ifndef PSS_MIN_CTAS64
#define PSS_MIN_CTAS64 1
#endif
// one-buffer passes whose next copy is issued from the last stage: at the
// start of a tile, ask for the next tile's data to be brought into L2, so
// that the copy reads L2 (column passes: one tensor prefetch; row passes:
// one bulk prefetch per row and input; measured at 4096^2: row pass
// 225 -> 220 us, 8192^2: 525 -> 509 us, 1024^2 unchanged)
#ifndef PSS_COL_PREFETCH
#define PSS_COL_PREFETCH 1
#endif
#ifndef PSS_ROW_PREFETCH
#define PSS_ROW_PREFETCH 1
#endif
// one-buffer column passes with an early copy store their tiles by tensor
// copy through a half-tile staging area (PSS_COL_HALF_STORE=0: strided stores)
#ifndef PSS_COL_HALF_STORE
#define PSS_COL_HALF_STORE 1
#endif
#ifndef PSS_MAX_NBUF64
#define PSS_MAX_NBUF64 2
#endif
template <class Rl> struct Shape {
    static constexpr int ESZ = 2 * int(sizeof(Rl));
    static constexpr int MIN_CTAS = sizeof(Rl) == 4 ? PSS_MIN_CTAS : PSS_MIN_CTAS64;
    static constexpr int MAX_NBUF = sizeof(Rl) == 4 ? PSS_MAX_NBUF : PSS_MAX_NBUF64;
    // points per thread of the row and column transforms
    static constexpr int RP = sizeof(Rl) == 4 ? PSS_ROW_P : PSS_ROW_P64;
    static constexpr int CP = sizeof(Rl) == 4 ? PSS_COL_P : PSS_COL_P64;
    // rows of at least PSS_BIG_N points may use PSS_ROW_P_BIG / PSS_COL_P_BIG
    static constexpr int RPB = sizeof(Rl) == 4 ? PSS_ROW_P_BIG : RP;
    static constexpr int CPB = sizeof(Rl) == 4 ? PSS_COL_P_BIG : CP;
    __host__ __device__ static constexpr int rowP(int n) { return n < RP ? n : n >= PSS_BIG_N ? RPB : RP; }
    __host__ __device__ static constexpr int colP(int n) { return n < CP ? n : n >= PSS_BIG_N ? CPB : CP; }
    // columns per tile: 64-byte row segments (FP32) when the thread budget
    // (PSS_COL_THREADS) and shared memory (nbuf buffers) allow.  With `wide`,
    // a tile whose row segments would drop below 32 bytes (one DRAM sector)
    // may use up to PSS_COL_WIDE_THREADS threads instead (measured on GB300,
    // NLS FP32: column pass +41 % at 4096^2 and +38 % at 8192^2; at 2048^2,
    // where 32-byte segments fit in 256 threads, the wider tile was slower)
    __host__ __device__ static constexpr int cols_capped(int n, int p, int nbuf, int cap)
    {
        int w = sizeof(Rl) == 4 ? PSS_COL_WMAX : 4;
        while (w > 1 && ((long)nbuf * w * (n + n / 16) * ESZ > 200 * 1024L || w * (n / p) > cap)) w /= 2;
        return w;
    }
    __host__ __device__ static constexpr int cols(int n, int p, int nbuf = 2, bool wide = false)
    {
        const int w = cols_capped(n, p, nbuf, PSS_COL_THREADS);
        return (wide && w * ESZ < 32) ? cols_capped(n, p, nbuf, PSS_COL_WIDE_THREADS) : w;
    }
};

// Launch-shape variants a lean FP32 pass is compiled in (the plan the
// autotuner picks from, per kernel instance): 0 = the shapes above (32 points
// per thread, two CTAs of <= 128 registers per SM); 1 = 16 points per thread,
// four CTAs per SM (<= 64 registers).
template <class Rl, int VAR> struct VarShape {
    static constexpr int PCAP = VAR == 1 ? 16 : 1 << 20;
    static constexpr int CTAS = VAR == 1 ? 4 : Shape<Rl>::MIN_CTAS;
    static constexpr int TPS = VAR == 1 ? 1024 : PSS_THREADS_PER_SM;
};
__host__ __device__ constexpr int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int imax(int a, int b) { return a > b ? a : b; }

// dynamic shared memory a pass may use per CTA (the GB300 limit is 227 KB)
constexpr size_t SMEM_LIMIT = 200 * 1024;

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

// LEAN: one shared-memory buffer and (FP32) two resident CTAs per SM, for ops
// whose transforms fit in 128 registers; otherwise a double buffer, one CTA.
template <class Rl, int N, int NIN, bool LEAN = false, int PMAX = 32, int VAR = 0> struct RowCfg {
    using VS = VarShape<Rl, VAR>;
    static constexpr int P = imin(imin(Shape<Rl>::rowP(N), PMAX), VS::PCAP);
    static constexpr int T = N / P;
    // ~256 threads per CTA; small rows (N <= 256) take ~64 so that a batch of
    // small grids still spreads over many SMs (a 128^2 field is 2 CTAs, not 1/2)
    static constexpr int RT = N <= 256 ? PSS_ROW_THREADS_SMALL : PSS_ROW_THREADS;
    static constexpr int ROWS = T >= RT ? 1 : RT / T;
    static constexpr int PADLOG = pad_log(P);
    static constexpr int LINE = N + (N >> PADLOG);
    static constexpr int THREADS = ROWS * T;
    // barrier of one row's threads (fft_sync): a warp, the CTA, or the row's
    // own named barrier when the CTA holds several multi-warp rows
    static constexpr int BLOCK = T <= 32 ? 0 : (ROWS > 1 ? T : 1);
    // two buffers of NIN input lines per row (one when two do not fit)
    static constexpr int BUF = NIN * ROWS * LINE;
    static constexpr int MAXB = LEAN ? Shape<Rl>::MAX_NBUF : 2;
    static constexpr int NBUF = (MAXB > 1 && size_t(2) * BUF * Shape<Rl>::ESZ <= SMEM_LIMIT) ? 2 : 1;
    static constexpr size_t SMEM = size_t(NBUF) * BUF * Shape<Rl>::ESZ;
    // resident CTAs the registers are budgeted for: at most VS::TPS threads
    // per SM (512: 128 registers each)
    static constexpr int MIN_CTAS =
        LEAN ? (THREADS * VS::CTAS <= VS::TPS ? VS::CTAS : (VS::TPS / THREADS > 1 ? VS::TPS / THREADS : 1)) : 1;
};

template <class Rl, int N, int NIN, bool LEAN = false, int PMAX = 32, int VAR = 0> struct ColCfg {
    using VS = VarShape<Rl, VAR>;
    static constexpr int P = imin(imin(Shape<Rl>::colP(N), PMAX), VS::PCAP);
    static constexpr int T = N / P;
    // lean ops (one buffer, <= 128 registers) may take the wide tiles
    static constexpr int W = LEAN ? Shape<Rl>::cols(N, P, NIN * Shape<Rl>::MAX_NBUF, true) : Shape<Rl>::cols(N, P);
    static constexpr int PADLOG = pad_log(P);
    static constexpr int STRIDE = col_stride(N + (N >> PADLOG), W, Shape<Rl>::ESZ);
    static constexpr int THREADS = W * T;
    static constexpr int BLOCK = THREADS > 32 ? 1 : 0;  // a column's threads span the CTA
    static constexpr int BUF = NIN * W * STRIDE;
    static constexpr int MAXB = LEAN ? Shape<Rl>::MAX_NBUF : 2;
    static constexpr int NBUF = (MAXB > 1 && size_t(2) * BUF * Shape<Rl>::ESZ <= SMEM_LIMIT) ? 2 : 1;
    static constexpr size_t SMEM = size_t(NBUF) * BUF * Shape<Rl>::ESZ;
    // resident CTAs the registers are budgeted for: at most VS::TPS threads
    // per SM (512: 128 registers each)
    static constexpr int MIN_CTAS =
        LEAN ? (THREADS * VS::CTAS <= VS::TPS ? VS::CTAS : (VS::TPS / THREADS > 1 ? VS::TPS / THREADS : 1)) : 1;
};

// points per thread an op allows at length N: Op::pmax(N) where the op
// defines it, else Op::PMAX
template <class Op, class = void> struct HasPmaxN : std::false_type {};
template <class Op> struct HasPmaxN<Op, std::void_t<decltype(Op::pmax(1))>> : std::true_type {};
template <class Op> __host__ __device__ constexpr int op_pmax(int n)
{
    if constexpr (HasPmaxN<Op>::value) return Op::pmax(n);
    else return Op::PMAX;
}
template <class Rl, int N, class Op, int VAR = 0>
using RowCfgOf = RowCfg<Rl, N, Op::NIN, Op::LEAN, op_pmax<Op>(N), VAR>;
template <class Rl, int N, class Op, int VAR = 0>
using ColCfgOf = ColCfg<Rl, N, Op::NIN, Op::LEAN, op_pmax<Op>(N), VAR>;

// ----------------------------------------------------------------------------
// cp.async: per-thread asynchronous global -> shared copies (no registers held)

template <int BYTES> __device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gmem_src), "n"(BYTES)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stage P points of a line (element t + T m at stride st) into a padded
// shared line at the same positions.
template <int P, int T, class V, class Sm>
__device__ __forceinline__ void stage_line(const Sm &sm, const V *__restrict__ src, int64_t st, int t)
{
    const V *p = src + int64_t(t) * st;  // running pointer: one live address
    const int64_t step = int64_t(T) * st;
#pragma unroll
    for (int m = 0; m < P; ++m, p += step) cp_async<sizeof(V)>(&sm[t + T * m], p);
}
template <int P, int T, class V, class Sm>
__device__ __forceinline__ void read_line(V (&v)[P], const Sm &sm, int t)
{
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = sm[t + T * m];
}

// ----------------------------------------------------------------------------
// Kernel shells

// An op may define prologue<N>(): work every thread of a CTA does once before
// the first tile (filling shared-memory tables); the kernel synchronises
// after it.
template <class Op, class = void> struct HasPrologue : std::false_type {};
template <class Op>
struct HasPrologue<Op, std::void_t<decltype(std::declval<const Op &>().template prologue<1024>())>>
    : std::true_type {};
template <int N, class Op> __device__ __forceinline__ void op_prologue(const Op &op)
{
    if constexpr (HasPrologue<Op>::value) op.template prologue<N>();
}

// An op that sets EARLY_NEXT takes a hook as the last argument of row() and
// calls it once its last transform has made its last shared-memory access
// (block_fft's hook): a single-buffered row pass then issues the copies of
// its next tile there, under the rest of the tile's arithmetic and stores.
template <class Op, class = void> struct EarlyNext : std::false_type {};
template <class Op>
struct EarlyNext<Op, std::void_t<decltype(Op::EARLY_NEXT)>> : std::integral_constant<bool, Op::EARLY_NEXT> {};

// rows_total = batch * ny; row r of the batch starts at element r * NX
template <class Rl, int N, class Op, int VAR>
__global__ void __launch_bounds__(RowCfgOf<Rl, N, Op, VAR>::THREADS, RowCfgOf<Rl, N, Op, VAR>::MIN_CTAS)
    k_row(Op op, const TW<Rl> *__restrict__ tw, int64_t rows_total)
{
    using C = RowCfgOf<Rl, N, Op, VAR>;
    using V = V2<Rl>;
    using Sm = SmemLine<V, C::PADLOG>;
    constexpr int NIN = Op::NIN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *const buf = reinterpret_cast<V *>(smem_raw);
    const int lr = threadIdx.x / C::T, t = threadIdx.x % C::T;
    const int64_t tiles = (rows_total + C::ROWS - 1) / C::ROWS;

    auto line = [&](int b, int k) { return Sm{buf + b * C::BUF + (k * C::ROWS + lr) * C::LINE}; };
    auto issue = [&](int64_t tile, int b) {
        const int64_t row = tile * C::ROWS + lr;
        if (tile < tiles && row < rows_total)
#pragma unroll
            for (int k = 0; k < NIN; ++k) stage_line<C::P, C::T>(line(b, k), op.in(k) + row * N, 1, t);
        cp_async_commit();
    };

    constexpr bool EARLY = EarlyNext<Op>::value && C::NBUF == 1;
    int64_t tile = blockIdx.x;
    if (C::NBUF == 2 || EARLY) issue(tile, 0);
    fill_stage_tw<N, C::P>(tw);
    op_prologue<N>(op);
    __syncthreads();
    for (int it = 0; tile < tiles; ++it, tile += gridDim.x) {
        int b = 0;
        if constexpr (C::NBUF == 2) {
            b = it & 1;
            issue(tile + gridDim.x, b ^ 1);
            cp_async_wait<1>();
        } else if constexpr (EARLY) {
            cp_async_wait<0>();  // issued during the previous tile (or above)
        } else {
            issue(tile, 0);
            cp_async_wait<0>();
        }
        const int64_t row = tile * C::ROWS + lr;
        V v[NIN][C::P];
        Sm sm[NIN];
#pragma unroll
        for (int k = 0; k < NIN; ++k) {
            sm[k] = line(b, k);
            read_line<C::P, C::T>(v[k], sm[k], t);
        }
        if constexpr (EARLY) {
            const int64_t next = tile + gridDim.x;
            if (PSS_ROW_PREFETCH && t == 0 && next < tiles && next * C::ROWS + lr < rows_total)
#pragma unroll
                for (int k = 0; k < NIN; ++k)
                    bulk_prefetch_l2(op.in(k) + (next * C::ROWS + lr) * N, unsigned(N * sizeof(V)));
            const auto hook = [&]() {
                fft_sync<C::BLOCK>();  // the row's last shared-memory reads are done
                issue(next, 0);
            };
            op.template row<N, C::P, C::BLOCK>(v, row, row < rows_total, t, sm, tw, hook);
        } else {
            op.template row<N, C::P, C::BLOCK>(v, row, row < rows_total, t, sm, tw);
            fft_sync<C::BLOCK>();  // this buffer is refilled by the next iteration's prefetch
        }
    }
    cp_async_wait<0>();
}

// input k of a column op: op.in(k, field) where the op chooses its source
// buffer per field, else op.in(k)
template <class Op, class = void> struct FieldIn : std::false_type {};
template <class Op>
struct FieldIn<Op, std::void_t<decltype(std::declval<const Op &>().in(0, int64_t(0)))>> : std::true_type {};
template <class Op> __device__ __forceinline__ auto col_in(const Op &op, int k, int64_t field)
{
    if constexpr (FieldIn<Op>::value) return op.in(k, field);
    else return op.in(k);
}

// Row stride of a column op's staged inputs: op.in_stride where the op
// defines it (inputs wider than the columns it visits), else nx.
template <class Op, class = void> struct HasInStride : std::false_type {};
template <class Op>
struct HasInStride<Op, std::void_t<decltype(std::declval<const Op &>().in_stride)>> : std::true_type {};
template <class Op> __host__ __device__ __forceinline__ int64_t in_stride(const Op &op, int64_t nx)
{
    if constexpr (HasInStride<Op>::value) return op.in_stride;
    else return nx;
}

// Column groups a column op visits: all nx / W of them, or, where the op
// defines skip_lo / skip_n, all but the skip_n groups from skip_lo on (a
// contiguous run the op knows to be zero and to stay zero).
template <class Op, class = void> struct SkipsGroups : std::false_type {};
template <class Op>
struct SkipsGroups<Op, std::void_t<decltype(std::declval<const Op &>().skip_n)>> : std::true_type {};
template <class Op> __host__ __device__ __forceinline__ int64_t kept_groups(const Op &op, int64_t groups)
{
    if constexpr (SkipsGroups<Op>::value) return groups - op.skip_n;
    else return groups;
}
template <class Op> __host__ __device__ __forceinline__ int64_t group_index(const Op &op, int64_t g)
{
    if constexpr (SkipsGroups<Op>::value) return g < op.skip_lo ? g : g + op.skip_n;
    else return g;
}

// tiles: (NX / W) column groups per field (fewer where the op skips some), fields in order
template <class Rl, int N, class Op, int VAR>
__global__ void __launch_bounds__(ColCfgOf<Rl, N, Op, VAR>::THREADS, ColCfgOf<Rl, N, Op, VAR>::MIN_CTAS)
    k_col(Op op, const TW<Rl> *__restrict__ tw, int64_t nx, int64_t batch)
{
    using C = ColCfgOf<Rl, N, Op, VAR>;
    using V = V2<Rl>;
    using Sm = SmemLine<V, C::PADLOG>;
    constexpr int NIN = Op::NIN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *const buf = reinterpret_cast<V *>(smem_raw);
    const int c = threadIdx.x % C::W, t = threadIdx.x / C::W;
    const int64_t groups = kept_groups(op, nx / C::W), tiles = groups * batch;

    auto line = [&](int b, int k) { return Sm{buf + b * C::BUF + (k * C::W + c) * C::STRIDE}; };
    auto issue = [&](int64_t tile, int b) {
        if (tile < tiles) {
            const int64_t field = tile / groups, x = group_index(op, tile % groups) * C::W + c;
#pragma unroll
            for (int k = 0; k < NIN; ++k)
                stage_line<C::P, C::T>(line(b, k), col_in(op, k, field) + field * N * in_stride(op, nx) + x,
                                       in_stride(op, nx), t);
        }
        cp_async_commit();
    };

    int64_t tile = blockIdx.x;
    if (C::NBUF == 2) issue(tile, 0);
    fill_stage_tw<N, C::P>(tw);
    op_prologue<N>(op);
    __syncthreads();
    for (int it = 0; tile < tiles; ++it, tile += gridDim.x) {
        int b = 0;
        if constexpr (C::NBUF == 2) {
            b = it & 1;
            issue(tile + gridDim.x, b ^ 1);
            cp_async_wait<1>();
        } else {
            issue(tile, 0);
            cp_async_wait<0>();
        }
        const int64_t field = tile / groups;
        const int x = int(group_index(op, tile % groups) * C::W + c);
        V v[NIN][C::P];
        Sm sm[NIN];
#pragma unroll
        for (int k = 0; k < NIN; ++k) {
            sm[k] = line(b, k);
            read_line<C::P, C::T>(v[k], sm[k], t);
        }
        op.template col<N, C::P, C::BLOCK>(v, field, x, t, sm, tw);
        fft_sync<C::BLOCK>();
    }
    cp_async_wait<0>();
}

// ----------------------------------------------------------------------------
// Column pass whose tiles arrive by one tensor copy each (see tma.cuh): for
// ops with one input array (the same for every field) that name a status
// word (op.status); the input's row stride and the skipped column groups
// follow in_stride() and group_index().  The tile lands as a dense [N][W] block at
// the start of the buffer; thread (c, t) reads its points t + T m of column c
// from there (a warp reads 32 consecutive points), and the padded column
// lines of the same buffer then serve as the transforms' exchange space (the
// first exchange store comes after a CTA barrier, so after every read).
template <class Op, class = void> struct TmaCol : std::false_type {};
template <class Op>
struct TmaCol<Op, std::void_t<decltype(std::declval<const Op &>().status)>>
    : std::integral_constant<bool, Op::NIN == 1 && !FieldIn<Op>::value> {};

// ops whose col() takes a hook for the start of the last stage of their last
// transform (COL_EARLY): the one-buffer column pass then issues the next
// tile's copy there.  PSS_COL_EARLY=0 compiles every op without it.
#ifndef PSS_COL_EARLY
#define PSS_COL_EARLY 1
#endif
template <class Op, class = void> struct ColEarly : std::false_type {};
template <class Op>
struct ColEarly<Op, std::void_t<decltype(Op::COL_EARLY)>> : std::integral_constant<bool, PSS_COL_EARLY && Op::COL_EARLY> {};

// dynamic shared memory of the tensor-copy column pass: the buffer, room to
// align it to 128 bytes and the mbarrier
template <class C> constexpr size_t tma_col_smem() { return C::SMEM + 128 + 16; }

// An op with COL_TMA_STORE = true whose output tile is its input tile (in
// place) lets the pass store its tiles by tensor copy: col<..., STORE = false>
// leaves the results in registers, the threads write them into shared memory
// as the dense [N][W] block of the input copy (or halves of it), and one
// thread stores that with one tensor copy in place of every thread's strided
// stores of 8-byte points.  The landing-buffer pass stages a tile in the
// group's exchange buffer; the one-buffer pass with an early copy, whose
// buffer then already receives the next tile, in a staging area of half a
// tile, stored in two halves (4096^2: 135 KB buffer + 64 KB staging).
template <class Op, class = void> struct TmaStoreOp : std::false_type {};
template <class Op>
struct TmaStoreOp<Op, std::void_t<decltype(Op::COL_TMA_STORE)>> : std::integral_constant<bool, Op::COL_TMA_STORE> {};

// the one-buffer pass's staging: on for an early-copy op that stores by tensor
// copy, where a column tile splits into two halves of whole row blocks
template <class Rl, int N, class Op> struct TmaHalfStore {
    using C = ColCfgOf<Rl, N, Op, 0>;
    static constexpr int R = N < 256 ? N : 256;
    // (one CTA per SM: the staging would not fit beside a second CTA)
    static constexpr bool ON = PSS_COL_HALF_STORE && TmaStoreOp<Op>::value && ColEarly<Op>::value &&
                               sizeof(Rl) == 4 && C::MIN_CTAS == 1 && N >= 512 && (N / R) % 2 == 0;
    static constexpr int HALF_BLOCKS = (N / R) / 2;  // row blocks of R rows per half
    static constexpr size_t BYTES = ON ? size_t(N / 2) * C::W * sizeof(V2<Rl>) : 0;
    static constexpr size_t SMEM = tma_col_smem<C>() + (ON ? 128 + BYTES : 0);
};


template <class Rl, int N, class Op>
__global__ void __launch_bounds__(ColCfgOf<Rl, N, Op, 0>::THREADS, ColCfgOf<Rl, N, Op, 0>::MIN_CTAS)
    k_col_tma(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap map_half, Op op,
              const TW<Rl> *__restrict__ tw, int64_t nx, int64_t batch, unsigned wait_limit, int skip_copy)
{
    using C = ColCfgOf<Rl, N, Op, 0>;
    using HS = TmaHalfStore<Rl, N, Op>;
    using V = V2<Rl>;
    using Sm = SmemLine<V, C::PADLOG>;
    static_assert(C::NBUF == 1, "one staging buffer");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // align to 128 bytes by an offset from the shared array itself (an
    // address rebuilt from an integer would lose the shared state space and
    // turn every exchange access into a generic one)
    const unsigned pad = (128u - (smem_addr(smem_raw) & 127u)) & 127u;
    V *const buf = reinterpret_cast<V *>(smem_raw + pad);
    const unsigned sbar = smem_addr(buf + C::BUF);
    // the half-tile staging area (HS::ON), 128-byte aligned after the mbarrier
    V *const stg = reinterpret_cast<V *>(smem_raw + pad + (size_t(C::BUF) * sizeof(V) + 16 + 127) / 128 * 128);
    const int c = threadIdx.x % C::W, t = threadIdx.x / C::W;
    // 32-bit tile counters (the launcher checks the count): fewer live registers
    const int groups = int(kept_groups(op, nx / C::W)), tiles = groups * int(batch);
    if (threadIdx.x == 0) mbar_init(sbar, 1);
    fill_stage_tw<N, C::P>(tw);
    op_prologue<N>(op);
    __syncthreads();
    // thread 0: ask for tile `tl` (the buffer's earlier shared-memory accesses
    // come first)
    auto issue = [&](int tl) {
        if (threadIdx.x != 0 || tl >= tiles) return;
        const int f = tl / groups;
        const int xs = int(group_index(op, tl - f * groups)) * C::W;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(sbar, unsigned(N * C::W * sizeof(V)));
        // skip_copy (host fault injection only): announce the bytes but start
        // no copy, so that the wait below runs out with nothing in flight
        if (!skip_copy) tma_load_4d(smem_addr(buf), &map, sbar, 2 * xs, 0, 0, f);
    };
    // an op with COL_EARLY calls a hook at the start of the last stage of its
    // last transform, after its last shared-memory access: the next tile's
    // copy is issued there and lands under that stage and the tile's stores
    constexpr bool EARLY = ColEarly<Op>::value;
    if (EARLY) issue(int(blockIdx.x));
    unsigned parity = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, parity ^= 1u) {
        const int field = tile / groups;
        const int x0 = int(group_index(op, tile - field * groups)) * C::W;
        if (!EARLY) issue(tile);
        const bool landed = mbar_wait(sbar, parity, wait_limit);
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) {
                atomicOr(op.status, STATUS_TMA_TIMEOUT);
                if (HS::ON) bulk_wait();  // this CTA's stores are done with the staging area
            }
            return;
        }
        V v[1][C::P];
#pragma unroll
        for (int m = 0; m < C::P; ++m) v[0][m] = buf[(t + C::T * m) * C::W + c];
        // an op with an early copy: the next tile into L2 now, so that its
        // copy, issued at the start of this tile's last stage, reads L2
        // (measured at 4096^2, NLS: column pass 279 -> 259 us; the ops that
        // copy at the tile's start were 3 % slower with it)
        if (EARLY && PSS_COL_PREFETCH && threadIdx.x == 0 && tile + int(gridDim.x) < tiles) {
            const int nt = tile + int(gridDim.x), nf = nt / groups;
            tma_prefetch_4d(&map, 2 * int(group_index(op, nt - nf * groups)) * C::W, 0, 0, nf);
        }
        const Sm sm[1] = {Sm{buf + c * C::STRIDE}};
        if constexpr (EARLY) {
            const int next = tile + int(gridDim.x);
            const auto hook = [&]() {
                fft_sync<C::BLOCK>();  // every shared-memory access of this tile is done
                issue(next);
            };
            if constexpr (HS::ON) {
                op.template col<N, C::P, C::BLOCK, Sm, decltype(hook), false>(v, int64_t(field), x0 + c, t, sm, tw,
                                                                               hook);
                // rows h N/2 + t + T m (m < P/2) of half h: its register m + h P/2
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (threadIdx.x == 0) bulk_wait_read();  // the staging area's last store has read it
                    __syncthreads();
#pragma unroll
                    for (int m = 0; m < C::P / 2; ++m) stg[(t + C::T * m) * C::W + c] = v[0][h * (C::P / 2) + m];
                    fence_proxy_async_smem();
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        tma_store_4d(&map_half, smem_addr(stg), 2 * x0, 0, h * HS::HALF_BLOCKS, field);
                        bulk_commit();
                    }
                }
            } else {
                op.template col<N, C::P, C::BLOCK>(v, int64_t(field), x0 + c, t, sm, tw, hook);
            }
        } else {
            op.template col<N, C::P, C::BLOCK>(v, int64_t(field), x0 + c, t, sm, tw);
            fft_sync<C::BLOCK>();  // every read of this tile is done before the next copy lands
        }
    }
    if (HS::ON && threadIdx.x == 0) bulk_wait();
}

// ----------------------------------------------------------------------------
// Column pass in two parts per tile, for ops whose tile work is long and whose
// tiles are few (Navier-Stokes at batch 1: 342 tiles of four 4096-point
// columns on 152 SMs, one tile per SM at a time, are 2.25 rounds, so the
// last third of the pass ran on a quarter of the SMs).  Work item i < tiles
// is part 0 of tile i (its tensor copy, then op.col_part(..., 0)); item
// tiles + i is part 1 (op.col_part(..., 1)), which reads what part 0 stored.
// CTAs claim positions in increasing order from a counter (op.claim, zero at
// launch); split_item maps them to items so that part 1 of a tile comes
// about one item's time after its part 0 (its stores are then done, and
// still in L2), and always after it.  So whenever a CTA holds part 1 of a
// tile, part 0 has been claimed by a running CTA, and part 0 never waits on
// another item: every wait ends.
// Part 0 publishes its stores (CTA barrier, fence, release store of the
// pass's epoch into the tile's word op.tile_done[i]); part 1 polls that word
// with acquire loads, bounded: if it never comes it sets STATUS_SPLIT_TIMEOUT
// and returns.  An op opts in with COL_SPLIT = true.
template <class Op, class = void> struct SplitOp : std::false_type {};
template <class Op>
struct SplitOp<Op, std::void_t<decltype(Op::COL_SPLIT)>> : std::integral_constant<bool, Op::COL_SPLIT> {};

__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// polls of a part-1 wait, 256 ns apart: about a second
constexpr unsigned SPLIT_WAIT_LIMIT = 1u << 22;

// Claim position p (0 <= p < 2 tiles) -> (part, tile), with a lag of `lag`
// tiles (1 <= lag <= tiles): part 0 of tiles 0 .. lag - 1, then part 0 of
// tile lag + j and part 1 of tile j alternately, then the last parts 1.
// Part 1 of tile j sits at lag + 2 j + 1, after part 0 of tile j (at j or
// at 2 j - lag < j + lag + 1).
__host__ __device__ __forceinline__ void split_item(int p, int tiles, int lag, int &part, int &tile)
{
    const int mixed = 2 * (tiles - lag);
    if (p < lag) {
        part = 0;
        tile = p;
    } else if (p < lag + mixed) {
        const int q = p - lag;
        part = q & 1;
        tile = part ? q >> 1 : lag + (q >> 1);
    } else {
        part = 1;
        tile = tiles - lag + (p - lag - mixed);
    }
}
constexpr int STATUS_SPLIT_TIMEOUT = 2;

template <class Rl, int N, class Op>
__global__ void __launch_bounds__(ColCfgOf<Rl, N, Op, 0>::THREADS, ColCfgOf<Rl, N, Op, 0>::MIN_CTAS)
    k_col_split(const __grid_constant__ CUtensorMap map, Op op, const TW<Rl> *__restrict__ tw, int64_t nx,
                int64_t batch, unsigned wait_limit, int skip_copy)
{
    using C = ColCfgOf<Rl, N, Op, 0>;
    using V = V2<Rl>;
    using Sm = SmemLine<V, C::PADLOG>;
    static_assert(C::NBUF == 1 && C::BLOCK == 1, "one staging buffer; transforms span the CTA");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *const buf = reinterpret_cast<V *>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));
    const unsigned sbar = smem_addr(buf + C::BUF);
    __shared__ int item_s;
    const int c = threadIdx.x % C::W, t = threadIdx.x / C::W;
    const int groups = int(kept_groups(op, nx / C::W)), tiles = groups * int(batch);
    const unsigned epoch = unsigned(*op.epoch) + 1u;
    if (threadIdx.x == 0) mbar_init(sbar, 1);
    fill_stage_tw<N, C::P>(tw);
    op_prologue<N>(op);
    __syncthreads();
    unsigned parity = 0;
    const int lag = imin(int(gridDim.x), tiles);
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(op.claim, 1);
        __syncthreads();
        const int pos = item_s;  // rewritten only after the barrier at the end of this item
        if (pos >= 2 * tiles) break;
        int part, tile;
        split_item(pos, tiles, lag, part, tile);
        const int field = tile / groups;
        const int x0 = int(group_index(op, tile - field * groups)) * C::W;
        const Sm sm[1] = {Sm{buf + c * C::STRIDE}};
        V v[1][C::P];
        if (part == 0) {
            if (threadIdx.x == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(sbar, unsigned(N * C::W * sizeof(V)));
                // skip_copy (host fault injection only): no copy is started
                if (!skip_copy) tma_load_4d(smem_addr(buf), &map, sbar, 2 * x0, 0, 0, field);
            }
            const bool landed = mbar_wait(sbar, parity, wait_limit);
            parity ^= 1u;
            if (__syncthreads_or(!landed)) {
                if (threadIdx.x == 0) atomicOr(op.status, STATUS_TMA_TIMEOUT);
                return;
            }
#pragma unroll
            for (int m = 0; m < C::P; ++m) v[0][m] = buf[(t + C::T * m) * C::W + c];
            op.template col_part<N, C::P, C::BLOCK>(v, int64_t(field), x0 + c, t, sm, tw, 0);
            __syncthreads();  // every store of part 0 has been made
            if (threadIdx.x == 0) {
                __threadfence();
                st_release_gpu(op.tile_done + tile, epoch);
            }
        } else {
            bool ok = true;
            if (threadIdx.x == 0) {
                ok = false;
                for (unsigned i = 0; i < SPLIT_WAIT_LIMIT; ++i) {
                    if (ld_acquire_gpu(op.tile_done + tile) == epoch) {
                        ok = true;
                        break;
                    }
                    __nanosleep(256);
                }
                __threadfence();
            }
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicOr(op.status, STATUS_SPLIT_TIMEOUT);
                return;
            }
            op.template col_part<N, C::P, C::BLOCK>(v, int64_t(field), x0 + c, t, sm, tw, 1);
        }
        fft_sync<C::BLOCK>();  // the buffer's readers are done before the next copy lands
    }
}

// ----------------------------------------------------------------------------
// Tensor-copy column pass whose copies overlap the transforms.  With one
// staging buffer (k_col_tma) a CTA asks for its next tile only when it has
// finished the current one, so every copy's latency is exposed to that CTA.
// Here a CTA holds two groups of C::THREADS threads (each the shape of one
// k_col_tma CTA), each with its own exchange buffer, and one landing buffer
// that the tiles arrive in (a dense [N][W] block).  The CTA's tiles k = 0, 1,
// 2, ... (blockIdx.x + k gridDim.x) go to group k mod 2.  A group waits for
// its tile in the landing buffer, reads it into registers and then at once
// asks for the other group's next tile into the landing buffer, so that
// copy lands while both groups compute; the transforms' exchanges use the
// group's own buffer.  Copies for group g complete on mbarrier g (a
// barrier's phases then follow one group's tiles, so their parities cannot
// be confused).  Each group synchronises on its own named barriers
// (fft_sync<THREADS>: ids 1 and 2; the votes below: ids 3 and 4), so the
// groups run independently.  An op opts in with COL_LAND = true (its
// exchanges must use fft_sync<BLOCK>, not CTA-wide barriers).
template <class Op, class = void> struct LandOp : std::false_type {};
template <class Op>
struct LandOp<Op, std::void_t<decltype(Op::COL_LAND)>> : std::integral_constant<bool, Op::COL_LAND> {};

// elements between the two groups' exchange buffers: a multiple of 128 bytes,
// so that each can be the aligned source of a tensor store
template <class C> constexpr int land_gbuf() { return (C::BUF * int(C::SMEM / C::BUF) + 127) / 128 * 128 / int(C::SMEM / C::BUF); }

// dynamic shared memory: two exchange buffers and the landing buffer, room to
// align them to 128 bytes, two mbarriers and the control words (abort flag,
// copies issued towards each group)
template <class C> constexpr size_t land_col_smem()
{
    return 2 * size_t(land_gbuf<C>()) * (C::SMEM / C::BUF) + size_t(C::T) * C::P * C::W * (C::SMEM / C::BUF) + 128 +
           16 + 16;
}

// OR of `v` over the G threads of this thread's group (named barrier id)
template <int G> __device__ __forceinline__ bool group_any(bool v, int id)
{
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"(unsigned(v)), "r"(id), "n"(G)
        : "memory");
    return r != 0;
}

// volatile 32-bit shared-memory word access (control words of k_col_land)
__device__ __forceinline__ int lds_vol(unsigned addr)
{
    int v;
    asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void sts_vol(unsigned addr, int v)
{
    asm volatile("st.volatile.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// mbar_wait that also gives up once the CTA's abort flag (at `abort`) is set
__device__ __forceinline__ bool mbar_wait_or_abort(unsigned bar, unsigned parity, unsigned limit, unsigned abort)
{
    for (unsigned i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (lds_vol(abort)) return false;
    }
    return false;
}

template <class Rl, int N, class Op>
__global__ void __launch_bounds__(2 * ColCfgOf<Rl, N, Op, 0>::THREADS,
                                  imax(1, PSS_THREADS_PER_SM / (2 * ColCfgOf<Rl, N, Op, 0>::THREADS)))
    k_col_land(const __grid_constant__ CUtensorMap map, Op op, const TW<Rl> *__restrict__ tw, int64_t nx,
               int64_t batch, unsigned wait_limit, int skip_copy)
{
    using C = ColCfgOf<Rl, N, Op, 0>;
    using V = V2<Rl>;
    using Sm = SmemLine<V, C::PADLOG>;
    constexpr int G = C::THREADS;  // threads per group
    static_assert(C::NBUF == 1 && G % 32 == 0 && 2 * G <= 1024, "two groups of one-buffer tiles");
    constexpr bool TST = TmaStoreOp<Op>::value;
    constexpr int GB = land_gbuf<C>();  // elements per group buffer (128-byte multiple)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *const xbuf = reinterpret_cast<V *>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));
    V *const land = xbuf + 2 * GB;                      // the dense [N][W] landing block
    const unsigned sbar = smem_addr(land + N * C::W);   // mbarrier of group g at sbar + 8 g
    const unsigned ctrl = sbar + 16;                    // [0] abort, [1 + g] copies issued towards group g
    const int grp = threadIdx.x / G, tg = threadIdx.x % G;
    const int c = tg % C::W, t = tg / C::W;
    const int groups = int(kept_groups(op, nx / C::W)), tiles = groups * int(batch);

    // one thread: ask for `tile` into the landing buffer, for group g
    auto issue = [&](int tile, int g) {
        if (tile >= tiles) return;
        const int field = tile / groups;
        const int x0 = int(group_index(op, tile - field * groups)) * C::W;
        fence_proxy_async_smem();  // the landing buffer's earlier reads come first
        mbar_arrive_expect_tx(sbar + 8 * g, unsigned(N * C::W * sizeof(V)));
        // skip_copy (host fault injection only): announce the bytes but start
        // no copy, so that the waits run out with nothing in flight
        if (!skip_copy) tma_load_4d(smem_addr(land), &map, sbar + 8 * g, 2 * x0, 0, 0, field);
        sts_vol(ctrl + 4 * (1 + g), lds_vol(ctrl + 4 * (1 + g)) + 1);
    };
    if (threadIdx.x == 0) {
        mbar_init(sbar, 1);
        mbar_init(sbar + 8, 1);
        sts_vol(ctrl, 0);
        sts_vol(ctrl + 4, 0);
        sts_vol(ctrl + 8, 0);
        issue(int(blockIdx.x), 0);
    }
    fill_stage_tw<N, C::P>(tw);
    op_prologue<N>(op);
    __syncthreads();

    const Sm sm[1] = {Sm{xbuf + grp * GB + c * C::STRIDE}};
    unsigned par = 0;
    for (int tile = int(blockIdx.x) + grp * int(gridDim.x); tile < tiles; tile += 2 * int(gridDim.x), par ^= 1u) {
        const bool landed = mbar_wait_or_abort(sbar + 8 * grp, par, wait_limit, ctrl);
        if (group_any<G>(!landed, 3 + grp)) {
            if (tg == 0) {
                atomicOr(op.status, STATUS_TMA_TIMEOUT);
                sts_vol(ctrl, 1);  // the other group stops at its next wait
                // leave no copy of this CTA in flight: wait (bounded) for the
                // last copy issued towards each group
                for (int g = 0; g < 2; ++g) {
                    const int n = lds_vol(ctrl + 4 * (1 + g));
                    if (n > 0) mbar_wait(sbar + 8 * g, unsigned(n - 1) & 1u, wait_limit);
                }
            }
            if (TST && tg == 0) bulk_wait();  // this group's stores are done with its buffer
            return;
        }
        // the group's previous tensor store has read its buffer before the
        // group's next exchange writes (a group barrier comes in between)
        if (TST && tg == 0) bulk_wait_read();
        V v[1][C::P];
#pragma unroll
        for (int m = 0; m < C::P; ++m) v[0][m] = land[(t + C::T * m) * C::W + c];
        fft_sync<G>();  // the group has read the landing buffer: refill it for the other group
        if (tg == 0) issue(tile + int(gridDim.x), grp ^ 1);
        const int field = tile / groups;
        const int x0 = int(group_index(op, tile - field * groups)) * C::W;
        if constexpr (TST) {
            op.template col<N, C::P, G, Sm, NoHook, false>(v, int64_t(field), x0 + c, t, sm, tw, NoHook{});
            V *const dense = xbuf + grp * GB;
            fft_sync<G>();  // the group's last exchange reads are done
#pragma unroll
            for (int m = 0; m < C::P; ++m) dense[(t + C::T * m) * C::W + c] = v[0][m];
            fence_proxy_async_smem();
            fft_sync<G>();
            if (tg == 0) {
                tma_store_4d(&map, smem_addr(dense), 2 * x0, 0, 0, field);
                bulk_commit();
            }
        } else {
            op.template col<N, C::P, G>(v, int64_t(field), x0 + c, t, sm, tw);
        }
    }
    if (TST && tg == 0) bulk_wait();
}

// ----------------------------------------------------------------------------
// Store helper: register m -> element t + T m of a line with stride st
template <int P, int T, class V>
__device__ __forceinline__ void store_line(const V (&v)[P], V *__restrict__ p, int64_t st, int t,
                                           bool ok)
{
    if (!ok) return;
    V *q = p + int64_t(t) * st;  // running pointer: one live address
    const int64_t step = int64_t(T) * st;
#pragma unroll
    for (int m = 0; m < P; ++m, q += step) *q = v[m];
}

// ----------------------------------------------------------------------------
// Plain transforms (the 2D FFT of every step, Section 4)

template <class Rl, int DIR> struct RowFft {
    static constexpr int NIN = 1;
    static constexpr bool LEAN = true;
    static constexpr int PMAX = 32;
    V2<Rl> *data;
    Rl scale;  // applied after the transform when != 1
    __device__ const V2<Rl> *in(int) const { return data; }
    template <int N, int P, int BLOCK, class Sm>
    __device__ __forceinline__ void row(V2<Rl> (&v)[1][P], int64_t r, bool ok, int t, const Sm (&sm)[1],
                                        const TW<Rl> *tw) const
    {
        block_fft<N, P, DIR, BLOCK>(v[0], sm[0], t, tw);
        if (scale != Rl(1))
#pragma unroll
            for (int m = 0; m < P; ++m) v[0][m] = cscale(v[0][m], scale);
        store_line<P, N / P>(v[0], data + r * N, 1, t, ok);
    }
};

template <class Rl, int DIR> struct ColFft {
    static constexpr int NIN = 1;
    static constexpr bool LEAN = true;
    static constexpr int PMAX = 32;
    V2<Rl> *data;
    int64_t nx;
    Rl scale;
    __device__ const V2<Rl> *in(int) const { return data; }
    template <int N, int P, int BLOCK, class Sm>
    __device__ __forceinline__ void col(V2<Rl> (&v)[1][P], int64_t field, int x, int t,
                                        const Sm (&sm)[1], const TW<Rl> *tw) const
    {
        block_fft<N, P, DIR, BLOCK>(v[0], sm[0], t, tw);
        if (scale != Rl(1))
#pragma unroll
            for (int m = 0; m < P; ++m) v[0][m] = cscale(v[0][m], scale);
        store_line<P, N / P>(v[0], data + field * N * nx + x, nx, t, true);
    }
};

}  // namespace pss
