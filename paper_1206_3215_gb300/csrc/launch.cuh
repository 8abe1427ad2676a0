// Dispatch from a run-time grid length to the compiled kernel shapes.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdlib>
#include <cstring>

#include "passes.cuh"
#include "plan.h"

namespace pss {

// Supported lengths of either grid axis.
#define PSS_FOR_EACH_N(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192)

// Allow a kernel `bytes` of dynamic shared memory, once per device
// (attributes belong to the device's context).  done_mask is a static of the
// caller, one per kernel instance.
template <class K>
inline cudaError_t allow_smem(K kernel, size_t bytes, std::atomic<unsigned> &done_mask)
{
    // the 48 KB a kernel has without opting in count its static shared
    // memory too, so any dynamic request opts in (once per device)
    if (bytes == 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned bit = 1u << (dev & 31);
    if (done_mask.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) done_mask.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// Persistent grid: as many CTAs as fit on the device at once (occupancy of
// this kernel instance, cached per device), never more than there are tiles.
template <class K> inline cudaError_t resident_ctas(K kernel, int threads, size_t smem,
                                                    int (&cache)[32], int *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int &c = cache[dev & 31];
    if (c == 0) {
        int per_sm = 0, sms = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem)) != cudaSuccess)
            return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        c = (per_sm > 0 ? per_sm : 1) * sms;
    }
    *out = c;
    return cudaSuccess;
}

template <class Rl, int N, class Op> constexpr bool tunable()
{
    return sizeof(Rl) == 4 && Op::LEAN && N >= 512 && !SkipsGroups<Op>::value;
}

inline int plan_pick(PlanSlot &slot)
{
    PlanTuning *pt = plan_tuning();
    if (pt->force >= 0) {
        const int kind = pt->open_kind;
        if (kind == 0 || kind == 1) {
            bool seen = false;
            for (int i = 0; i < pt->nused[kind]; ++i) seen = seen || pt->used[kind][i] == &slot;
            if (!seen && pt->nused[kind] < 8) pt->used[kind][pt->nused[kind]++] = &slot;
        }
        return pt->force;
    }
    // PSS_PLAN=0|1 pins every tunable kernel to one variant (read per launch)
    const char *e = getenv("PSS_PLAN");
    if (e && (e[0] == '0' || e[0] == '1') && e[1] == 0) return e[0] - '0';
    const int v = slot.var.load(std::memory_order_acquire);
    return v < 0 ? 0 : v;
}

template <class Rl, int N, class Op, int VAR>
inline cudaError_t launch_row_v(Op op, const TW<Rl> *tw, int64_t rows_total, cudaStream_t s)
{
    using C = RowCfgOf<Rl, N, Op, VAR>;
    auto k = k_row<Rl, N, Op, VAR>;
    static std::atomic<unsigned> done{0};
    static int ctas[32] = {};
    cudaError_t e = allow_smem(k, C::SMEM, done);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (rows_total + C::ROWS - 1) / C::ROWS;
    if (tiles <= 0) return cudaSuccess;
    int grid = 0;
    if ((e = resident_ctas(k, C::THREADS, C::SMEM, ctas, &grid)) != cudaSuccess) return e;
    if (tiles < grid) grid = int(tiles);
    k<<<dim3(unsigned(grid)), C::THREADS, C::SMEM, s>>>(op, tw, rows_total);
    return cudaGetLastError();
}

template <class Rl, int N, class Op, int VAR>
inline cudaError_t launch_col_v(Op op, const TW<Rl> *tw, int64_t nx, int64_t batch, cudaStream_t s)
{
    using C = ColCfgOf<Rl, N, Op, VAR>;
    auto k = k_col<Rl, N, Op, VAR>;
    static std::atomic<unsigned> done{0};
    static int ctas[32] = {};
    cudaError_t e = allow_smem(k, C::SMEM, done);
    if (e != cudaSuccess) return e;
    const int64_t tiles = kept_groups(op, nx / C::W) * batch;
    if (tiles <= 0) return cudaSuccess;
    int grid = 0;
    if ((e = resident_ctas(k, C::THREADS, C::SMEM, ctas, &grid)) != cudaSuccess) return e;
    if (tiles < grid) grid = int(tiles);
    k<<<dim3(unsigned(grid)), C::THREADS, C::SMEM, s>>>(op, tw, nx, batch);
    return cudaGetLastError();
}

// PSS_TMA=0 stages column tiles with per-point cp.async copies instead of
// tensor copies (read per launch)
inline bool tma_enabled()
{
    const char *e = getenv("PSS_TMA");
    return !(e && e[0] == '0' && e[1] == 0);
}

template <class Rl, int N, class Op> constexpr bool tma_col()
{
    using C = ColCfgOf<Rl, N, Op, 0>;
    return TmaCol<Op>::value && sizeof(Rl) == 4 && C::BLOCK && C::NBUF == 1 && N >= 256 &&
           (C::W * sizeof(V2<Rl>)) % 16 == 0;
}

template <class Rl, int N, class Op>
inline cudaError_t launch_col_tma(Op op, const TW<Rl> *tw, int64_t nx, int64_t batch, cudaStream_t s)
{
    using C = ColCfgOf<Rl, N, Op, 0>;
    using HS = TmaHalfStore<Rl, N, Op>;
    auto k = k_col_tma<Rl, N, Op>;
    constexpr size_t smem = HS::SMEM;
    static std::atomic<unsigned> done{0};
    static int ctas[32] = {};
    cudaError_t e = allow_smem(k, smem, done);
    if (e != cudaSuccess) return e;
    const int64_t tiles = kept_groups(op, nx / C::W) * batch;
    if (tiles <= 0) return cudaSuccess;
    if (tiles > INT32_MAX - 2 * 65536) return cudaErrorInvalidValue;  // the kernel counts tiles in 32 bits
    CUtensorMap map, map_half;
    if ((e = encode_col_map(&map, op.in(0), int(sizeof(V2<Rl>)), in_stride(op, nx), N, batch, C::W)) != cudaSuccess)
        return e;
    // the half-tile store box (the op writes its input array in place)
    if constexpr (HS::ON) {
        if ((e = encode_col_map(&map_half, op.in(0), int(sizeof(V2<Rl>)), in_stride(op, nx), N, batch, C::W, 2)) !=
            cudaSuccess)
            return e;
    } else {
        map_half = map;
    }
    int grid = 0;
    if ((e = resident_ctas(k, C::THREADS, smem, ctas, &grid)) != cudaSuccess) return e;
    if (tiles < grid) grid = int(tiles);
    // PSS_FAULT=tma_timeout: the tile copies are announced but not started and
    // the wait is short, so every CTA gives up, sets the status word and
    // returns (a bounded wait that runs out; nothing is left in flight)
    const char *f = getenv("PSS_FAULT");
    const bool inject = f && strcmp(f, "tma_timeout") == 0;
    k<<<dim3(unsigned(grid)), C::THREADS, smem, s>>>(map, map_half, op, tw, nx, batch, inject ? 64u : TMA_WAIT_LIMIT,
                                                      inject ? 1 : 0);
    return cudaGetLastError();
}

// PSS_COL_LAND=0 keeps the one-buffer tensor-copy column pass for ops that
// opted into the landing-buffer one (read per launch)
inline bool land_enabled()
{
    const char *e = getenv("PSS_COL_LAND");
    return !(e && e[0] == '0' && e[1] == 0);
}

// the landing-buffer column pass: an op that opted in, two groups within the
// per-SM thread budget the registers are planned for, the buffers and the
// stage twiddles within the 227 KB of shared memory a CTA may have
template <class Rl, int N, class Op> constexpr bool land_col()
{
    using C = ColCfgOf<Rl, N, Op, 0>;
    return tma_col<Rl, N, Op>() && LandOp<Op>::value && 2 * C::THREADS <= PSS_THREADS_PER_SM &&
           land_col_smem<C>() + 16 * size_t(StageTw<N, C::P>::COUNT) <= 227 * 1024;
}

template <class Rl, int N, class Op>
inline cudaError_t launch_col_land(Op op, const TW<Rl> *tw, int64_t nx, int64_t batch, cudaStream_t s)
{
    using C = ColCfgOf<Rl, N, Op, 0>;
    auto k = k_col_land<Rl, N, Op>;
    constexpr size_t smem = land_col_smem<C>();
    static std::atomic<unsigned> done{0};
    static int ctas[32] = {};
    cudaError_t e = allow_smem(k, smem, done);
    if (e != cudaSuccess) return e;
    const int64_t tiles = kept_groups(op, nx / C::W) * batch;
    if (tiles <= 0) return cudaSuccess;
    if (tiles > INT32_MAX - 2 * 65536) return cudaErrorInvalidValue;  // the kernel counts tiles in 32 bits
    CUtensorMap map;
    if ((e = encode_col_map(&map, op.in(0), int(sizeof(V2<Rl>)), in_stride(op, nx), N, batch, C::W)) != cudaSuccess)
        return e;
    int grid = 0;
    if ((e = resident_ctas(k, 2 * C::THREADS, smem, ctas, &grid)) != cudaSuccess) return e;
    if (tiles < grid) grid = int(tiles);
    const char *f = getenv("PSS_FAULT");
    const bool inject = f && strcmp(f, "tma_timeout") == 0;
    k<<<dim3(unsigned(grid)), 2 * C::THREADS, smem, s>>>(map, op, tw, nx, batch, inject ? 64u : TMA_WAIT_LIMIT,
                                                          inject ? 1 : 0);
    return cudaGetLastError();
}

// PSS_COL_SPLIT=0 keeps the one-part column pass for ops that opted into the
// split one (read per launch)
inline bool split_enabled()
{
    const char *e = getenv("PSS_COL_SPLIT");
    return !(e && e[0] == '0' && e[1] == 0);
}

// the split column pass: an op that opted in, in the one-buffer shapes
// (where the landing-buffer pass does not fit)
template <class Rl, int N, class Op> constexpr bool split_col()
{
    return tma_col<Rl, N, Op>() && SplitOp<Op>::value && ColCfgOf<Rl, N, Op, 0>::BLOCK == 1 &&
           !land_col<Rl, N, Op>();
}

template <class Rl, int N, class Op>
inline cudaError_t launch_col_split(Op op, const TW<Rl> *tw, int64_t nx, int64_t batch, cudaStream_t s)
{
    using C = ColCfgOf<Rl, N, Op, 0>;
    auto k = k_col_split<Rl, N, Op>;
    constexpr size_t smem = tma_col_smem<C>();
    static std::atomic<unsigned> done{0};
    static int ctas[32] = {};
    cudaError_t e = allow_smem(k, smem, done);
    if (e != cudaSuccess) return e;
    const int64_t tiles = kept_groups(op, nx / C::W) * batch;
    if (tiles <= 0) return cudaSuccess;
    // the kernel counts items (two per tile) and claims them in 32 bits
    if (tiles > (INT32_MAX - 2 * 65536) / 2) return cudaErrorInvalidValue;
    CUtensorMap map;
    if ((e = encode_col_map(&map, op.in(0), int(sizeof(V2<Rl>)), in_stride(op, nx), N, batch, C::W)) != cudaSuccess)
        return e;
    int grid = 0;
    if ((e = resident_ctas(k, C::THREADS, smem, ctas, &grid)) != cudaSuccess) return e;
    if (2 * tiles < grid) grid = int(2 * tiles);
    const char *f = getenv("PSS_FAULT");
    const bool inject = f && strcmp(f, "tma_timeout") == 0;
    k<<<dim3(unsigned(grid)), C::THREADS, smem, s>>>(map, op, tw, nx, batch, inject ? 64u : TMA_WAIT_LIMIT,
                                                      inject ? 1 : 0);
    return cudaGetLastError();
}

template <class Rl, int N, class Op>
inline cudaError_t launch_row_n(Op op, const TW<Rl> *tw, int64_t rows_total, cudaStream_t s)
{
    if constexpr (tunable<Rl, N, Op>()) {
        static PlanSlot slot;
        // every tile width divides the row stride: a variant choice needs no caller change
        if (plan_pick(slot) == 1) return launch_row_v<Rl, N, Op, 1>(op, tw, rows_total, s);
    }
    return launch_row_v<Rl, N, Op, 0>(op, tw, rows_total, s);
}

template <class Rl, int N, class Op>
inline cudaError_t launch_col_n(Op op, const TW<Rl> *tw, int64_t nx, int64_t batch, cudaStream_t s)
{
    if constexpr (tunable<Rl, N, Op>()) {
        static PlanSlot slot;
        if (nx % ColCfgOf<Rl, N, Op, 1>::W == 0 && plan_pick(slot) == 1)
            return launch_col_v<Rl, N, Op, 1>(op, tw, nx, batch, s);
    }
    if constexpr (land_col<Rl, N, Op>())
        if (tma_enabled() && land_enabled()) return launch_col_land<Rl, N, Op>(op, tw, nx, batch, s);
    if constexpr (split_col<Rl, N, Op>())
        if (tma_enabled() && split_enabled()) return launch_col_split<Rl, N, Op>(op, tw, nx, batch, s);
    if constexpr (tma_col<Rl, N, Op>())
        if (tma_enabled()) return launch_col_tma<Rl, N, Op>(op, tw, nx, batch, s);
    return launch_col_v<Rl, N, Op, 0>(op, tw, nx, batch, s);
}

// Row pass over every row of a [batch][ny][nx] array: transform length nx.
template <class Rl, class Op>
inline cudaError_t launch_row(int64_t nx, Op op, const TW<Rl> *tw, int64_t rows_total, cudaStream_t s)
{
    switch (nx) {
#define PSS_CASE(N) \
    case N: return launch_row_n<Rl, N>(op, tw, rows_total, s);
        PSS_FOR_EACH_N(PSS_CASE)
#undef PSS_CASE
    default: return cudaErrorInvalidValue;
    }
}

// Column pass over every column of a [batch][ny][nx] array: transform length ny.
template <class Rl, class Op>
inline cudaError_t launch_col(int64_t ny, int64_t nx, Op op, const TW<Rl> *tw, int64_t batch,
                              cudaStream_t s)
{
    switch (ny) {
#define PSS_CASE(N) \
    case N: return launch_col_n<Rl, N>(op, tw, nx, batch, s);
        PSS_FOR_EACH_N(PSS_CASE)
#undef PSS_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pss
