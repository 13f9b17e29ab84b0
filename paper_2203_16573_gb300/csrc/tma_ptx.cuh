// tma_ptx.cuh -- inline-PTX wrappers of the tensor memory accelerator and
// shared-memory mbarriers used by the TMA-fed phase kernels (stencil_tma.cu,
// stencil_march.cu): barrier set-up, expected-byte arrival, bounded waits,
// tensor-map prefetch and 2-D tile copies global -> shared.
#pragma once
#include <cuda.h>

#include "stencil_impl.cuh"

namespace ssx {
namespace {

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for phase `parity` of the barrier to complete, at most timeout_ns
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity,
                                          unsigned long long timeout_ns) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try(bar, parity))
        if (globaltimer() - t0 > timeout_ns) return false;
    return true;
}
// fetch a tensor map into the descriptor cache ahead of its first copy (a hint)
__device__ __forceinline__ void prefetch_map(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(map)) : "memory");
}
// 2-D tile copy global -> shared, completion counted on the mbarrier
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// The next tile >= tile on this CTA's stride whose sweep steps in launch t
// (total if none); *jo = its sweep. Every thread computes it (uniform).
template <class JobT>
__device__ __forceinline__ int next_active(const JobT *__restrict__ jobs, int njobs, int total,
                                           int t, int tile, int G, int *jo) {
    while (tile < total) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {   // last sweep whose tile_base <= tile
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&jobs[mid].job.tile_base) <= tile) lo = mid; else hi = mid - 1;
        }
        const int st = t - __ldg(&jobs[lo].job.offset);
        if (st >= 0 && st < __ldg(&jobs[lo].job.nt)) {
            *jo = lo;
            return tile;
        }
        const int end = __ldg(&jobs[lo].job.tile_base) + __ldg(&jobs[lo].job.tiles);
        tile += (end - tile + G - 1) / G * G;   // skip the rest of an idle sweep
    }
    *jo = 0;
    return total;
}

}  // namespace
}  // namespace ssx
