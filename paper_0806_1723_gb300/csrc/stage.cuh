// Plane staging shared by the staged kernels (stage.cu, mg.cu): bulk copies of contiguous node
// runs into shared memory with completion counted on mbarriers, bounded waits, L2 prefetches.
#pragma once
#include "internal.cuh"

namespace lasto {
namespace stage {

constexpr unsigned long long SG_WAIT_NS = 2000000000ull;

struct StageGeom {
    int tiles_j;      // ceil((ny - 2) / rows per tile)
    int chunk;        // planes per block
    unsigned oslot;   // floats per other-colour slot (a multiple of 4)
    unsigned bslot;   // floats per right-hand-side slot
    int hx1;          // (nx - 1) / 2 rounded up to a multiple of 4: x coefficients per parity
};

__device__ __forceinline__ uint32_t sg_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sg_now()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// true once the phase of the given parity has completed; false after SG_WAIT_NS
__device__ __forceinline__ bool sg_wait(uint32_t bar, uint32_t parity)
{
    uint64_t t0 = 0;
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        const uint64_t t = sg_now();
        if (t0 == 0)
            t0 = t;
        else if (t - t0 > SG_WAIT_NS)
            return false;
    }
}

// [start, start + len) in floats from the array base: both ends multiples of 4 (16 bytes), the
// end clipped to the last whole 16 bytes of the N-node array (the up to 3 nodes past it are the
// last nodes of the face plane's last row, which no interior update reads)
__device__ __forceinline__ void sg_range(unsigned a, unsigned e, unsigned N, unsigned& start, unsigned& len)
{
    start = a & ~3u;
    e = min((e + 3u) & ~3u, N & ~3u);
    len = e > start ? e - start : 0u;
}

// the other colour's run of plane p: rows j0 - 1 .. j0 + nr (the tile's rows and one on each side)
__device__ __forceinline__ void sg_orange(const LevelT<float>& L, int c, int p, int j0, int nr, unsigned& start,
                                          unsigned& len)
{
    const unsigned nxy = (unsigned)L.nx * (unsigned)L.ny;
    const unsigned lo = (unsigned)p * nxy + (unsigned)(j0 - 1) * (unsigned)L.nx;
    const unsigned hi = (unsigned)p * nxy + (unsigned)(j0 + nr + 1) * (unsigned)L.nx - 1u;
    const unsigned h0 = (unsigned)(1 - c) * L.H;
    sg_range(h0 + (lo >> 1), h0 + (hi >> 1) + 1u, (unsigned)L.N(), start, len);
}

// the colour's own run of plane p (right-hand side): rows j0 .. j0 + nr - 1
__device__ __forceinline__ void sg_brange(const LevelT<float>& L, int c, int p, int j0, int nr, unsigned& start,
                                          unsigned& len)
{
    const unsigned nxy = (unsigned)L.nx * (unsigned)L.ny;
    const unsigned lo = (unsigned)p * nxy + (unsigned)j0 * (unsigned)L.nx;
    const unsigned hi = (unsigned)p * nxy + (unsigned)(j0 + nr) * (unsigned)L.nx - 1u;
    const unsigned h0 = (unsigned)c * L.H;
    sg_range(h0 + (lo >> 1), h0 + (hi >> 1) + 1u, (unsigned)L.N(), start, len);
}

// the same run brought into L2 only (no completion to wait for)
__device__ __forceinline__ void sg_prefetch(const float* src, unsigned start, unsigned len)
{
    if (len) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src + start), "r"(len * 4u) : "memory");
}

// one bulk copy of len floats from src + start into the slot, counted on bar
__device__ __forceinline__ void sg_issue(const float* src, unsigned start, unsigned len, float* slot, uint32_t bar)
{
    // the slot's previous contents were read through the generic proxy (ordered before this by
    // the block barrier); the copy writes through the async proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(len * 4u) : "memory");
    if (len)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                sg_smem(slot)),
            "l"(src + start), "r"(len * 4u), "r"(bar)
            : "memory");
}

}  // namespace stage
}  // namespace lasto
