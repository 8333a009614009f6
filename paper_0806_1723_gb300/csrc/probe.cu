// Arithmetic throughput probes (chains of fused multiply-adds on every SM, in FP64 or FP32)
// and the self-test of the bounded device waits.
//
// The method has no counterpart; these measure the ceilings the roofline fractions of the
// ALU-bound kernels are stated against (the plain FP64 smoother and the FP32-pair density
// deposit), on the chip and clock the kernels themselves run on.  Each thread runs
// PROBE_CHAINS independent chains a <- a * m + c (m slightly below one, so the values stay
// finite and normal) and writes their sum, so nothing can be folded away.  Work per launch:
// 2 * PROBE_CHAINS * iters FLOP per thread.
#include "internal.cuh"

namespace lasto {

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(int iters, T* __restrict__ out)
{
    const int t = blockIdx.x * PROBE_THREADS + threadIdx.x;
    const T m = T(0.9999990463256836), c = T(1e-3);
    T a[PROBE_CHAINS];
#pragma unroll
    for (int q = 0; q < PROBE_CHAINS; q++) a[q] = T(1) + T(q) * T(0.125) + T(t & 7) * T(0.01);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < 16; r++)
#pragma unroll
            for (int q = 0; q < PROBE_CHAINS; q++) a[q] = fma(a[q], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int q = 0; q < PROBE_CHAINS; q++) s += a[q];
    out[t] = s;
}

__device__ __forceinline__ uint64_t probe_now()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Self-test of the bounded wait the staged tensor-core kernels use: one thread waits on an
// mbarrier that nothing arrives at, polling try_wait against %globaltimer; after limit_ns it
// gives up and raises LASTO_ERR_TIMEOUT in *status, as those kernels do.  No copy is in
// flight and no tensor memory is held, so the kernel then simply returns.
__global__ void k_wait_selftest(unsigned long long limit_ns, int* status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    const uint64_t t0 = probe_now();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(b), "r"(0u)
            : "memory");
        if (ok) return;
        if (probe_now() - t0 > limit_ns) break;
    }
    atomicMax(status, (int)LASTO_ERR_TIMEOUT);
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned long long limit_ns, int* status, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(limit_ns, status);
    return cudaGetLastError();
}

cudaError_t launch_fma_probe(int precision, int blocks, int iters, void* out, cudaStream_t s)
{
    if (blocks < 1 || iters < 1 || !out) return cudaErrorInvalidValue;
    if (precision == 0)
        k_fma_probe<double><<<blocks, PROBE_THREADS, 0, s>>>(iters, static_cast<double*>(out));
    else
        k_fma_probe<float><<<blocks, PROBE_THREADS, 0, s>>>(iters, static_cast<float*>(out));
    return cudaGetLastError();
}

}  // namespace lasto
