// Tensor-memory-accelerator staging for the column passes (sm_103a).
//
// A column tile is W adjacent columns of one field: N row segments of W
// complex points, one segment per row of the [batch][ny][nx] array.  Staged
// point by point, every thread issues one small copy per point it owns and a
// warp's copy touches 32/W separate segments; one cp.async.bulk.tensor copy
// instead moves the whole tile into shared memory as a dense [N][W] block and
// signals an mbarrier with the byte count when it has landed.
//
// The array is described to the copy engine as a 4D tensor of 4- or 8-byte
// reals (a complex point is two of them):
//   dim 0: 2 nx reals of a row (contiguous),
//   dim 1: R rows (stride one row),
//   dim 2: ny / R blocks of R rows,
//   dim 3: batch fields,
// with R = min(ny, 256) because no box extent may exceed 256.  A box of
// {2 W, R, ny / R, 1} at coordinates {2 x0, 0, 0, field} is the column tile
// starting at column x0.  Copies start on a 16-byte boundary: 2 x0 reals of
// 4 (8) bytes with x0 a multiple of W, and W * 8 (16) bytes a multiple of 16.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pss {

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    // make the initialised barrier visible to the copy engine
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// arrive (one of the barrier's expected arrivals) and announce `bytes` of
// transactions that complete this phase
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Wait until the phase with the given parity has completed.  try_wait
// suspends for a bounded, hardware-defined time per call; after `limit`
// unsuccessful calls the wait gives up and returns false.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, unsigned limit)
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
    }
    return false;
}

// order this thread's earlier generic-proxy shared-memory accesses (made
// visible to it by a CTA barrier) before later copy-engine accesses
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 4D tiled copy global -> shared; completion is counted on `bar`
__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap *map, unsigned bar, int c0, int c1,
                                            int c2, int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// Ask for the 4D box at these coordinates to be brought into L2 (no shared
// memory, no completion to wait for): a later copy of the box then reads L2
__device__ __forceinline__ void tma_prefetch_4d(const CUtensorMap *map, int c0, int c1, int c2, int c3)
{
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}
// the same for `bytes` (a multiple of 16) contiguous bytes from p (16-byte aligned)
__device__ __forceinline__ void bulk_prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// 4D tiled copy shared -> global of one box (the same tensor map and
// coordinates as the load of that box), tracked in this thread's bulk-async
// group; the source must be 128-byte aligned and its writes made visible to
// the copy engine first (fence_proxy_async_smem by the writers, then a barrier)
__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, unsigned src, int c0, int c1, int c2, int c3)
{
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(src), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// until this thread's committed stores have read their shared-memory source
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// until they have completed
__device__ __forceinline__ void bulk_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// iterations of mbar_wait before a tile copy counts as lost (each try_wait
// call may itself suspend for a while: this is seconds, not cycles)
constexpr unsigned TMA_WAIT_LIMIT = 1u << 24;

// Status word a pass kernel sets when a copy wait ran out (the pass then
// returns without finishing its tiles); read and cleared by the host.
constexpr int STATUS_TMA_TIMEOUT = 1;

// Host: the column-tile tensor map of a [batch][ny][nx] complex array of
// element size esz (8: complex64, 16: complex128), for tiles of w columns;
// with parts > 1 the box is 1/parts of a column tile tall (its row blocks
// start at block (ny / R / parts) h for part h).
cudaError_t encode_col_map(CUtensorMap *map, const void *base, int esz, int64_t nx, int64_t ny, int64_t batch,
                           int w, int parts = 1);

}  // namespace pss
