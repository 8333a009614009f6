// Interstitial overlap and Hamiltonian contributions (Section 3, Eq. 3.11-3.14, grid-point
// form) of a Slater-type basis over the nodes outside every atom sphere:
//   S_ab = sum_P phi_a(P) phi_b(P) Vol(P),
//   H_ab = 1/2 sum_P (phi_a(P) phi~_b(P) + phi~_a(P) phi_b(P)) Vol(P),
// phi_a = r^(n-1) e^{-zeta r} y_lm about its atom (Eq. 3.13), written r^(n-1-l) e^{-zeta r} S_lm(d)
// with the solid harmonic S_lm, and phi~_a = [-1/2 Lap + V] phi_a =
// 1/2 [(l(l+1) - n(n-1)) r^(n-3) + 2 zeta n r^(n-2) - zeta^2 r^(n-1)] e^{-zeta r} y_lm + V phi_a
// (Eq. 3.14).  Vol(P) is the node's dual-cell volume.  Functions are atom-major, then in the
// basis table's order, m = -l..l.
//
// Stages: (1) the interstitial nodes are listed in grid order (count, scan, scatter) with
// sqrt(Vol); (2) per chunk of listed nodes, tables A[p][f] = sqrt(Vol) phi_f and
// T[p][f] = sqrt(Vol) phi~_f (FP32, functions padded with zeros to the tile width); (3) a
// contraction over the upper-triangle function tiles, S = A^T A and 2H = A^T T + T^T A, either
// on the tensor cores (3 x TF32, below) or in FP32 SIMT arithmetic, partial sums added in FP64
// and node ranges meeting by FP64 atomic addition; (4) the lower triangle is mirrored.
#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace lasto {

namespace {

constexpr int HS_T = 64;       // functions per tile side
constexpr int HS_KC = 32;      // nodes per step
constexpr int HS_NT = 256;     // contraction threads: 16 x 16, each a 4 x 4 block
constexpr int HS_MAXB = 8;     // basis table entries
constexpr int HS_MAXF = 64;    // functions per atom
constexpr int HS_CNT = 1024;   // nodes per compaction block
constexpr size_t HS_TABLE_BYTES = (size_t)2 << 30;   // both tables of one chunk

struct MonoF32 {
    float coef;
    unsigned char a, b, c, pad;
};

__constant__ MonoF32 c_hs_mono[N_MONO_TERMS];   // grouped by lm
__constant__ int c_hs_first[NLM + 1];            // terms of lm: [first[lm], first[lm+1])

std::mutex g_hs_mutex;
int g_hs_device = -1;

cudaError_t ensure_hs_tables()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_hs_mutex);
    if (g_hs_device == dev) return cudaSuccess;
    std::vector<Mono> t(N_MONO_TERMS);
    host_monomials(t.data());
    std::vector<MonoF32> o;
    int first[NLM + 1];
    for (int lm = 0; lm < NLM; lm++) {
        first[lm] = (int)o.size();
        for (const Mono& m : t)
            if (m.lm == lm)
                o.push_back(MonoF32{(float)m.coef, (unsigned char)m.a, (unsigned char)m.b, (unsigned char)m.c, 0});
    }
    first[NLM] = (int)o.size();
    e = cudaMemcpyToSymbol(c_hs_mono, o.data(), sizeof(MonoF32) * o.size());
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_hs_first, first, sizeof(first));
    if (e == cudaSuccess) g_hs_device = dev;
    return e;
}

struct HsBasis {
    int per;                        // functions per atom
    int n[HS_MAXB], l[HS_MAXB];
    float zeta[HS_MAXB];
    unsigned char q_of[HS_MAXF];    // function within an atom -> table entry
    signed char m_of[HS_MAXF];      // -> m
};

struct HsGrid {
    int nx, ny, nz, na;
    const double *x, *y, *z, *pos, *R;
};

__device__ __forceinline__ bool hs_inside(const HsGrid& g, int i, int j, int k)
{
    for (int a = 0; a < g.na; a++) {
        const double dx = g.x[i] - g.pos[3 * a], dy = g.y[j] - g.pos[3 * a + 1], dz = g.z[k] - g.pos[3 * a + 2];
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        if (sqrt(d2) < g.R[a]) return true;
    }
    return false;
}

__device__ __forceinline__ double hs_dual(const double* c, int n, int q)
{
    return q == 0 ? 0.5 * (c[1] - c[0]) : q == n - 1 ? 0.5 * (c[n - 1] - c[n - 2]) : 0.5 * (c[q + 1] - c[q - 1]);
}

// block-wide exclusive scan of one int per thread; total = the block's sum
__device__ __forceinline__ int block_excl_scan(int v, int* warp_tot, int& total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    __syncthreads();
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    int before = 0;
    total = 0;
    for (int q = 0; q < nw; q++) {
        if (q < w) before += warp_tot[q];
        total += warp_tot[q];
    }
    return before + inc - v;
}

// (1a) interstitial nodes per block of HS_CNT nodes
__global__ void __launch_bounds__(256) k_hs_count(HsGrid g, int* __restrict__ cnt)
{
    __shared__ int wt[8];
    const size_t N = (size_t)g.nx * g.ny * g.nz;
    int c = 0;
    for (int e = 0; e < HS_CNT / 256; e++) {
        const size_t P = (size_t)blockIdx.x * HS_CNT + e * 256 + threadIdx.x;
        if (P < N) {
            const int i = (int)(P % g.nx), j = (int)((P / g.nx) % g.ny), k = (int)(P / ((size_t)g.nx * g.ny));
            c += !hs_inside(g, i, j, k);
        }
    }
    int total;
    block_excl_scan(c, wt, total);
    if (threadIdx.x == 0) cnt[blockIdx.x] = total;
}

// (1b) exclusive scan of the block counts (one block); off[nblk] = the number of listed nodes
__global__ void __launch_bounds__(1024) k_hs_scan(int nblk, const int* __restrict__ cnt, int* __restrict__ off)
{
    __shared__ int wt[32];
    int carry = 0;
    for (int b0 = 0; b0 < nblk; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        const int v = b < nblk ? cnt[b] : 0;
        int total;
        const int ex = block_excl_scan(v, wt, total);
        if (b < nblk) off[b] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) off[nblk] = carry;
}

// (1c) list the interstitial nodes of each block in grid order, with sqrt(Vol)
__global__ void __launch_bounds__(256) k_hs_scatter(HsGrid g, const int* __restrict__ off, int* __restrict__ idx,
                                                    float* __restrict__ sw)
{
    __shared__ int wt[8];
    const size_t N = (size_t)g.nx * g.ny * g.nz;
    int base = off[blockIdx.x];
    for (int e = 0; e < HS_CNT / 256; e++) {
        const size_t P = (size_t)blockIdx.x * HS_CNT + e * 256 + threadIdx.x;
        int i = 0, j = 0, k = 0, f = 0;
        if (P < N) {
            i = (int)(P % g.nx);
            j = (int)((P / g.nx) % g.ny);
            k = (int)(P / ((size_t)g.nx * g.ny));
            f = !hs_inside(g, i, j, k);
        }
        int total;
        const int ex = block_excl_scan(f, wt, total);
        if (f) {
            const double vol = hs_dual(g.x, g.nx, i) * hs_dual(g.y, g.ny, j) * hs_dual(g.z, g.nz, k);
            idx[base + ex] = (int)P;
            sw[base + ex] = (float)sqrt(vol);
        }
        base += total;
    }
}

__device__ __forceinline__ float hs_solid(int lm, float x, float y, float z)
{
    float s = 0.0f;
    for (int t = c_hs_first[lm]; t < c_hs_first[lm + 1]; t++) {
        const MonoF32 m = c_hs_mono[t];
        float v = m.coef;
        for (int p = 0; p < m.a; p++) v *= x;
        for (int p = 0; p < m.b; p++) v *= y;
        for (int p = 0; p < m.c; p++) v *= z;
        s += v;
    }
    return s;
}

// (2) tables of one chunk: rows p in [0, K) (listed nodes p0 + p; rows past n_list are zero),
// columns f in [0, Mp) (zero past M)
__global__ void __launch_bounds__(256) k_hs_basis(HsBasis B, HsGrid g, int M, int Mp, const int* __restrict__ idx,
                                                  const float* __restrict__ sw, const double* __restrict__ V,
                                                  int p0, int n_list, int K, float* __restrict__ A,
                                                  float* __restrict__ T)
{
    const size_t total = (size_t)K * Mp;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(e / Mp), f = (int)(e % Mp);
        float phi = 0.0f, tld = 0.0f;
        if (f < M && p0 + p < n_list) {
            const int P = idx[p0 + p];
            const int i = P % g.nx, j = (P / g.nx) % g.ny, k = P / (g.nx * g.ny);
            const int at = f / B.per, loc = f - at * B.per;
            const int q = B.q_of[loc], m = B.m_of[loc], n = B.n[q], l = B.l[q];
            const float zt = B.zeta[q];
            const float dx = (float)(g.x[i] - g.pos[3 * at]), dy = (float)(g.y[j] - g.pos[3 * at + 1]),
                        dz = (float)(g.z[k] - g.pos[3 * at + 2]);
            const float r = sqrtf(dx * dx + dy * dy + dz * dz);
            float rad = expf(-zt * r);
            for (int t = 0; t < n - 1 - l; t++) rad *= r;   // r^(n-1-l) e^{-zeta r}
            const float ir = 1.0f / r;
            const float kin =
                0.5f * ((float)(l * (l + 1) - n * (n - 1)) * ir * ir + 2.0f * zt * (float)n * ir - zt * zt);
            const float ps = sw[p0 + p] * rad * hs_solid(l * l + l + m, dx, dy, dz);
            phi = ps;
            tld = (kin + (float)V[P]) * ps;
        }
        A[e] = phi;
        T[e] = tld;
    }
}

__device__ __forceinline__ void hs_tile_of(int t, int nT, int& I, int& J)
{
    I = 0;
    while (t >= nT - I) {
        t -= nT - I;
        I++;
    }
    J = I + t;
}

// (3) FP32 SIMT contraction of upper-triangle tile (I <= J) over table rows [k0, k1)
__global__ void __launch_bounds__(HS_NT) k_hs_gemm_f32(int M, int Mp, int nT, const float* __restrict__ A,
                                                       const float* __restrict__ T, int kper, int K,
                                                       double* __restrict__ S, double* __restrict__ H2)
{
    __shared__ __align__(16) float sAI[HS_KC][HS_T], sTI[HS_KC][HS_T], sAJ[HS_KC][HS_T], sTJ[HS_KC][HS_T];
    int I, J;
    hs_tile_of(blockIdx.x, nT, I, J);
    const int k0 = blockIdx.y * kper, k1 = min(K, k0 + kper);
    if (k0 >= k1) return;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    double dS[4][4], dH[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) dS[i][j] = dH[i][j] = 0.0;
    for (int c = k0; c < k1; c += HS_KC) {
        __syncthreads();
        for (int e = tid; e < HS_KC * (HS_T / 4); e += HS_NT) {
            const int r = e / (HS_T / 4), c4 = (e % (HS_T / 4)) * 4;
            const size_t row = (size_t)(c + r) * Mp;
            *reinterpret_cast<float4*>(&sAI[r][c4]) = *reinterpret_cast<const float4*>(A + row + I * HS_T + c4);
            *reinterpret_cast<float4*>(&sTI[r][c4]) = *reinterpret_cast<const float4*>(T + row + I * HS_T + c4);
            *reinterpret_cast<float4*>(&sAJ[r][c4]) = *reinterpret_cast<const float4*>(A + row + J * HS_T + c4);
            *reinterpret_cast<float4*>(&sTJ[r][c4]) = *reinterpret_cast<const float4*>(T + row + J * HS_T + c4);
        }
        __syncthreads();
        float cS[4][4], cH[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) cS[i][j] = cH[i][j] = 0.0f;
#pragma unroll 8
        for (int kk = 0; kk < HS_KC; kk++) {
            const float4 a = *reinterpret_cast<const float4*>(&sAI[kk][ty * 4]);
            const float4 t = *reinterpret_cast<const float4*>(&sTI[kk][ty * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&sAJ[kk][tx * 4]);
            const float4 u = *reinterpret_cast<const float4*>(&sTJ[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, tv[4] = {t.x, t.y, t.z, t.w};
            const float bv[4] = {b.x, b.y, b.z, b.w}, uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    cS[i][j] = fmaf(av[i], bv[j], cS[i][j]);
                    cH[i][j] = fmaf(av[i], uv[j], fmaf(tv[i], bv[j], cH[i][j]));
                }
        }
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                dS[i][j] += (double)cS[i][j];
                dH[i][j] += (double)cH[i][j];
            }
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int a = I * HS_T + ty * 4 + i, b = J * HS_T + tx * 4 + j;
            if (a < M && b < M && a <= b) {
                atomicAdd(S + (size_t)a * M + b, dS[i][j]);
                atomicAdd(H2 + (size_t)a * M + b, dH[i][j]);
            }
        }
}

// (3') The same contraction on the fifth-generation tensor cores: tcgen05.mma kind::tf32 with
// 128 x 128 function tiles (M = N = 128, K = 8 nodes per MMA) and FP32 accumulators in tensor
// memory.  Each FP32 table value x is split into x_hi = x rounded to TF32 (10 stored mantissa
// bits) and x_lo = x - x_hi rounded to TF32; a product is formed as hi*hi + hi*lo + lo*hi
// (the dropped lo*lo is below 2^-21 of it), so S takes 3 MMAs per K step and 2H = A_I T_J^T +
// T_I A_J^T takes 6, all accumulating into two 128-column tensor-memory regions.
//
// A work unit is one upper-triangle tile and one segment of HS_SEG table rows; units are
// numbered segment-major so that the CTAs running at one time read the same table rows (which
// stay in L2).  A CTA's 256 threads produce the operands of a 16-node stage (thread m, h: row
// m, nodes 8h .. 8h+7) from the FP32 tables into a ring of three shared-memory stages in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix; the two K halves
// of an MMA 128 bytes apart, 8-row groups 256 bytes apart), the next stage's table values
// already loaded into registers; one thread issues the stage's 18 MMAs and commits them to the
// stage's mbarrier, which frees the stage.  Every HS_IV nodes the accumulation moves to the
// other pair of tensor-memory regions while the finished pair is read (tcgen05.ld) and added
// into the CTA's FP64 partial sums in global memory; at the end of a unit the partial sums go
// to S and 2H by FP64 atomic addition.  Every mbarrier wait is bounded; on a timeout the CTA
// records an error, stops issuing, waits (bounded) for its last MMAs, frees its tensor memory
// and returns.
constexpr int TC_TM = 128;                         // functions per tile side (MMA M and N)
constexpr int TC_NT = 256;                         // threads
constexpr int TC_SK = 16;                          // nodes per stage
constexpr int TC_RING = 3;                         // stages in shared memory
constexpr int TC_SLOT = TC_TM * TC_SK * 4;         // one operand of one stage: 8 KB
constexpr int TC_STAGE = 8 * TC_SLOT;              // A_I, T_I, A_J, T_J, each hi and lo
constexpr int TC_SMEM = TC_RING * TC_STAGE + 128;  // + alignment slack
constexpr int HS_IV = 512;                         // nodes per FP32 accumulation interval
constexpr int HS_SEG = 4096;                       // nodes per work unit
constexpr long long TC_SPIN = 1LL << 20;

__device__ __forceinline__ uint32_t hs_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// round to TF32 (nearest, ties away from zero, on the magnitude)
__device__ __forceinline__ float tf32_round(float v)
{
    return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ uint64_t hs_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;   // leading byte offset: the second K half
    d |= (uint64_t)(256 >> 4) << 32;   // stride byte offset: the next 8-row group
    d |= (uint64_t)1 << 46;
    return d;
}

// FP32 accumulator, TF32 A and B, both K-major, M = N = 128
constexpr uint32_t HS_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_TM >> 3) << 17) |
                              ((uint32_t)(TC_TM >> 4) << 24);

__device__ __forceinline__ uint64_t hs_now()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait on an mbarrier phase: false after about two seconds
__device__ __forceinline__ bool hs_wait(uint32_t mbar, uint32_t parity)
{
    uint64_t t0 = 0;
    for (long long it = 0; it < TC_SPIN; it++) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        const uint64_t t = hs_now();
        if (t0 == 0)
            t0 = t;
        else if (t - t0 > 2000000000ull)
            return false;
    }
    return false;
}

__device__ __forceinline__ void hs_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(HS_IDESC), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void hs_tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

struct HsUnit {
    int I, J, k0, k1;
};

__device__ __forceinline__ HsUnit hs_unit(int u, int pairs, int nT, int K)
{
    HsUnit w;
    const int seg = u / pairs;
    hs_tile_of(u - seg * pairs, nT, w.I, w.J);
    w.k0 = seg * HS_SEG;
    w.k1 = min(K, w.k0 + HS_SEG);
    return w;
}

__global__ void __launch_bounds__(TC_NT, 1) k_hs_gemm_tc(int M, int Mp, int nT, const float* __restrict__ A,
                                                        const float* __restrict__ T, int K, int units,
                                                        double* __restrict__ S, double* __restrict__ H2,
                                                        double* __restrict__ part, int* __restrict__ err)
{
    extern __shared__ unsigned char hs_dyn[];
    unsigned char* ring = reinterpret_cast<unsigned char*>(((uintptr_t)hs_dyn + 127) & ~(uintptr_t)127);
    __shared__ __align__(8) unsigned long long mbar[TC_RING];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = tid & (TC_TM - 1), h = tid >> 7;         // operand row, stage half
    const int q = warp & 3, cb = (warp >> 2) * TC_TM;      // drain: lane quarter, S or H columns
    const int pairs = nT * (nT + 1) / 2;
    double* mypart = part + (size_t)blockIdx.x * 2 * TC_TM * TC_TM;

    if (tid == 0) {
        for (int s = 0; s < TC_RING; s++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(hs_smem_u32(&mbar[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(
                         hs_smem_u32(&tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // table values of one stage for this thread: 4 arrays x 8 nodes
    auto load_stage = [&](const HsUnit& w, int row0, float (&v)[4][8]) {
        const size_t base = (size_t)(row0 + 8 * h) * Mp;
        const int cI = w.I * TC_TM + m, cJ = w.J * TC_TM + m;
#pragma unroll
        for (int kk = 0; kk < 8; kk++) {
            const size_t r = base + (size_t)kk * Mp;
            v[0][kk] = __ldg(A + r + cI);
            v[1][kk] = __ldg(T + r + cI);
            v[2][kk] = __ldg(A + r + cJ);
            v[3][kk] = __ldg(T + r + cJ);
        }
    };
    // drain the accumulator pair `set` into the partial sums (store on a unit's first interval)
    auto drain = [&](int set, bool first) {
        const uint32_t ta = tmem + (uint32_t)(set * 2 * TC_TM + cb) + ((uint32_t)(32 * q) << 16);
        const int row = 32 * q + lane;
        for (int c = 0; c < TC_TM; c += 16) {
            float v[16];
            hs_tmem_ld16(ta + (uint32_t)c, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; j++) {
                double* p = mypart + (size_t)(cb + c + j) * TC_TM + row;
                *p = first ? (double)v[j] : *p + (double)v[j];
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    };
    auto flush = [&](const HsUnit& w) {
        const int row = 32 * q + lane;
        const int a = w.I * TC_TM + row;
        double* dst = cb ? H2 : S;
        if (a >= M) return;
        for (int c = 0; c < TC_TM; c++) {
            const int b = w.J * TC_TM + c;
            if (b < M && a <= b) atomicAdd(dst + (size_t)a * M + b, mypart[(size_t)(cb + c) * TC_TM + row]);
        }
    };

    // a failed wait sets `fail` in its thread; the stage barriers combine the flags
    // (__syncthreads_or), so that every thread stops at the same point
    bool fail = false, stop = false;
    int g = 0;            // stages issued by this CTA
    int ic = 0;           // intervals started by this CTA
    // the interval whose accumulators wait to be drained
    bool pend = false, pend_first = false, pend_last = false;
    int pend_set = 0, pend_stage = 0;
    HsUnit pend_unit{0, 0, 0, 0};
    float vc[4][8], vn[4][8];

    for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
        const HsUnit w = hs_unit(u, pairs, nT, K);
        load_stage(w, w.k0, vc);
        for (int c0 = w.k0; c0 < w.k1 && !stop; c0 += HS_IV) {
            const int c1 = min(w.k1, c0 + HS_IV);
            const int set = ic & 1;
            const uint32_t tS = tmem + (uint32_t)(set * 2 * TC_TM), tH = tS + TC_TM;
            for (int r0 = c0; r0 < c1; r0 += TC_SK) {
                const int slot = g % TC_RING;
                const bool more = r0 + TC_SK < w.k1;
                if (more) load_stage(w, r0 + TC_SK, vn);
                if (g >= TC_RING && !hs_wait(hs_smem_u32(&mbar[slot]), (uint32_t)((g / TC_RING - 1) & 1)))
                    fail = true;
                unsigned char* st = ring + (size_t)slot * TC_STAGE;
#pragma unroll
                for (int x = 0; x < 4; x++) {
                    unsigned char* hi = st + (2 * x) * TC_SLOT + h * (TC_SLOT / 2) + (m >> 3) * 256 + (m & 7) * 16;
                    unsigned char* lo = hi + TC_SLOT;
#pragma unroll
                    for (int kq = 0; kq < 2; kq++) {
                        float4 H4, L4;
                        float* hp = &H4.x;
                        float* lp = &L4.x;
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            const float v = vc[x][4 * kq + e];
                            const float vh = tf32_round(v);
                            hp[e] = vh;
                            lp[e] = tf32_round(v - vh);
                        }
                        *reinterpret_cast<float4*>(hi + kq * 128) = H4;
                        *reinterpret_cast<float4*>(lo + kq * 128) = L4;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                if (__syncthreads_or(fail)) {
                    stop = true;
                    break;
                }
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t sb = hs_smem_u32(st);
#pragma unroll
                    for (int ks = 0; ks < 2; ks++) {
                        const uint32_t o = (uint32_t)(ks * (TC_SLOT / 2));
                        const uint64_t aIh = hs_desc(sb + 0 * TC_SLOT + o), aIl = hs_desc(sb + 1 * TC_SLOT + o);
                        const uint64_t tIh = hs_desc(sb + 2 * TC_SLOT + o), tIl = hs_desc(sb + 3 * TC_SLOT + o);
                        const uint64_t aJh = hs_desc(sb + 4 * TC_SLOT + o), aJl = hs_desc(sb + 5 * TC_SLOT + o);
                        const uint64_t tJh = hs_desc(sb + 6 * TC_SLOT + o), tJl = hs_desc(sb + 7 * TC_SLOT + o);
                        const uint32_t acc = (r0 > c0 || ks > 0) ? 1u : 0u;
                        hs_mma(tS, aIh, aJh, acc);
                        hs_mma(tS, aIh, aJl, 1u);
                        hs_mma(tS, aIl, aJh, 1u);
                        hs_mma(tH, aIh, tJh, acc);
                        hs_mma(tH, aIh, tJl, 1u);
                        hs_mma(tH, aIl, tJh, 1u);
                        hs_mma(tH, tIh, aJh, 1u);
                        hs_mma(tH, tIh, aJl, 1u);
                        hs_mma(tH, tIl, aJh, 1u);
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                            hs_smem_u32(&mbar[slot]))
                        : "memory");
                }
                // the previous interval's accumulators, once its last MMAs are done
                if (pend) {
                    // warp-uniform, since tcgen05.ld is a whole-warp instruction
                    const bool ok = hs_wait(hs_smem_u32(&mbar[pend_stage % TC_RING]), (uint32_t)((pend_stage / TC_RING) & 1));
                    if (!__all_sync(0xffffffffu, ok))
                        fail = true;
                    else {
                        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                        drain(pend_set, pend_first);
                        if (pend_last) flush(pend_unit);
                    }
                    pend = false;
                }
                g++;
                if (more) {
#pragma unroll
                    for (int x = 0; x < 4; x++)
#pragma unroll
                        for (int kk = 0; kk < 8; kk++) vc[x][kk] = vn[x][kk];
                }
            }
            if (stop) break;
            pend = true;
            pend_first = c0 == w.k0;
            pend_last = c1 == w.k1;
            pend_set = set;
            pend_stage = g - 1;
            pend_unit = w;
            ic++;
        }
    }
    if (pend && !stop) {
        const bool ok = hs_wait(hs_smem_u32(&mbar[pend_stage % TC_RING]), (uint32_t)((pend_stage / TC_RING) & 1));
        if (!__all_sync(0xffffffffu, ok))
            fail = true;
        else {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            drain(pend_set, pend_first);
            if (pend_last) flush(pend_unit);
        }
    }
    if (__syncthreads_or(fail)) {
        // let the MMAs already issued finish before the tensor memory is released
        if (tid == 0 && g > 0) hs_wait(hs_smem_u32(&mbar[(g - 1) % TC_RING]), (uint32_t)(((g - 1) / TC_RING) & 1));
        if (tid == 0 && err) atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem) : "memory");
}

// (4) S[b][a] = S[a][b] and H = H2 / 2 on both sides (the a <= b entries hold the sums)
__global__ void k_hs_mirror(int M, double* __restrict__ S, double* __restrict__ H)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= (size_t)M * M) return;
    const int a = (int)(t / M), b = (int)(t % M);
    if (a > b) return;
    const double h = 0.5 * H[t];
    H[t] = h;
    if (a < b) {
        S[(size_t)b * M + a] = S[t];
        H[(size_t)b * M + a] = h;
    }
}

size_t hs_rows_per_chunk(size_t N, int Mp)
{
    const size_t K = HS_TABLE_BYTES / (2 * sizeof(float) * (size_t)Mp) / HS_KC * HS_KC;
    return std::max<size_t>(HS_KC, std::min(K, (N + HS_KC - 1) / HS_KC * HS_KC));
}

int hs_sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

int g_hs_attr_device = -1;

cudaError_t ensure_hs_attributes()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_hs_mutex);
    if (g_hs_attr_device == dev) return cudaSuccess;
    e = cudaFuncSetAttribute(k_hs_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e == cudaSuccess) g_hs_attr_device = dev;
    return e;
}

}  // namespace

int hs_basis_check(int nb, const int* bn, const int* bl, const double* bz, int* per_out)
{
    if (nb < 1 || nb > HS_MAXB || !bn || !bl || !bz) return LASTO_ERR_INVALID_ARG;
    int per = 0;
    for (int q = 0; q < nb; q++) {
        if (bl[q] < 0 || bl[q] > 4 || bn[q] < bl[q] + 1 || bn[q] > 16 || !(bz[q] > 0.0)) return LASTO_ERR_INVALID_ARG;
        per += 2 * bl[q] + 1;
    }
    if (per > HS_MAXF) return LASTO_ERR_INVALID_ARG;
    *per_out = per;
    return LASTO_OK;
}

size_t hs_scratch_bytes(const int n[3], int M)
{
    const size_t N = (size_t)n[0] * n[1] * n[2];
    const size_t nblk = (N + HS_CNT - 1) / HS_CNT;
    const int Mp = (M + TC_TM - 1) / TC_TM * TC_TM;   // the larger padding of the two contractions
    const size_t K = hs_rows_per_chunk(N, Mp);
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    return up(sizeof(int) * nblk) + up(sizeof(int) * (nblk + 1)) + up(sizeof(int) * N) + up(sizeof(float) * N) +
           2 * up(sizeof(float) * (size_t)Mp * K) + up(sizeof(double) * 2 * TC_TM * TC_TM * (size_t)hs_sm_count()) +
           up(sizeof(int));
}

// scratch: hs_scratch_bytes(n, M) bytes, 256-byte aligned; carved into the block counts,
// offsets, listed nodes, sqrt(Vol), the two tables, the tensor-core CTAs' FP64 partial sums
// and an error flag.  Synchronises the stream twice (the number of listed nodes sizes the
// chunk loop; the error flag is read at the end).
int launch_interstitial_hs(const int n[3], const double* x, const double* y, const double* z, int na,
                           const double* pos, const double* R, int nb, const int* bn, const int* bl,
                           const double* bz, const double* V, double* S, double* H, void* scratch, int mode,
                           cudaStream_t s)
{
    int per = 0;
    if (hs_basis_check(nb, bn, bl, bz, &per) != LASTO_OK) return LASTO_ERR_INVALID_ARG;
    if (mode < LASTO_HS_DEFAULT || mode > LASTO_HS_TENSOR) return LASTO_ERR_INVALID_ARG;
    const bool tensor = mode != LASTO_HS_SIMT;
    HsBasis B{};
    B.per = per;
    for (int q = 0, f = 0; q < nb; q++) {
        B.n[q] = bn[q];
        B.l[q] = bl[q];
        B.zeta[q] = (float)bz[q];
        for (int m = -bl[q]; m <= bl[q]; m++, f++) {
            B.q_of[f] = (unsigned char)q;
            B.m_of[f] = (signed char)m;
        }
    }
    if (ensure_hs_tables() != cudaSuccess || ensure_hs_attributes() != cudaSuccess) return LASTO_ERR_CUDA;
    const int sms = hs_sm_count();
    if (sms < 1) return LASTO_ERR_CUDA;
    const int M = na * per;
    const int tile = tensor ? TC_TM : HS_T;
    const int Mp = (M + tile - 1) / tile * tile;
    const int nT = Mp / tile;
    const size_t N = (size_t)n[0] * n[1] * n[2];
    const int nblk = (int)((N + HS_CNT - 1) / HS_CNT);
    const size_t Kmax = hs_rows_per_chunk(N, (M + TC_TM - 1) / TC_TM * TC_TM);
    char* base = reinterpret_cast<char*>(scratch);
    auto carve = [&](size_t bytes) {
        char* p = base;
        base += (bytes + 255) / 256 * 256;
        return p;
    };
    int* cnt = reinterpret_cast<int*>(carve(sizeof(int) * nblk));
    int* off = reinterpret_cast<int*>(carve(sizeof(int) * (nblk + 1)));
    int* idx = reinterpret_cast<int*>(carve(sizeof(int) * N));
    float* sw = reinterpret_cast<float*>(carve(sizeof(float) * N));
    float* A = reinterpret_cast<float*>(carve(sizeof(float) * Mp * Kmax));
    float* T = reinterpret_cast<float*>(carve(sizeof(float) * Mp * Kmax));
    double* part = reinterpret_cast<double*>(carve(sizeof(double) * 2 * TC_TM * TC_TM * (size_t)sms));
    int* err = reinterpret_cast<int*>(carve(sizeof(int)));

    const HsGrid g{n[0], n[1], n[2], na, x, y, z, pos, R};
    cudaError_t e = cudaMemsetAsync(S, 0, sizeof(double) * (size_t)M * M, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(H, 0, sizeof(double) * (size_t)M * M, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e != cudaSuccess) return LASTO_ERR_CUDA;
    k_hs_count<<<nblk, 256, 0, s>>>(g, cnt);
    k_hs_scan<<<1, 1024, 0, s>>>(nblk, cnt, off);
    k_hs_scatter<<<nblk, 256, 0, s>>>(g, off, idx, sw);
    int n_list = 0;
    e = cudaMemcpyAsync(&n_list, off + nblk, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return LASTO_ERR_CUDA;

    const int pairs = nT * (nT + 1) / 2;
    for (int p0 = 0; p0 < n_list; p0 += (int)Kmax) {
        const int K = (int)std::min<size_t>(Kmax, ((size_t)(n_list - p0) + HS_KC - 1) / HS_KC * HS_KC);
        const size_t tot = (size_t)K * Mp;
        const unsigned gb = (unsigned)std::min<size_t>((tot + 255) / 256, (size_t)sms * 16);
        k_hs_basis<<<gb, 256, 0, s>>>(B, g, M, Mp, idx, sw, V, p0, n_list, K, A, T);
        if (tensor) {
            const int units = pairs * ((K + HS_SEG - 1) / HS_SEG);
            const int grid = std::min(units, sms);
            k_hs_gemm_tc<<<grid, TC_NT, TC_SMEM, s>>>(M, Mp, nT, A, T, K, units, S, H, part, err);
        } else {
            // node ranges per tile: about eight CTAs per SM in all
            int split = std::max(1, (8 * sms + pairs - 1) / pairs);
            split = std::min(split, K / HS_KC);
            const int kper = (K / HS_KC + split - 1) / split * HS_KC;
            split = (K + kper - 1) / kper;
            k_hs_gemm_f32<<<dim3((unsigned)pairs, (unsigned)split), HS_NT, 0, s>>>(M, Mp, nT, A, T, kper, K, S, H);
        }
    }
    k_hs_mirror<<<(unsigned)(((size_t)M * M + 255) / 256), 256, 0, s>>>(M, S, H);
    if (cudaGetLastError() != cudaSuccess) return LASTO_ERR_CUDA;
    int flag = 0;
    e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return LASTO_ERR_CUDA;
    return flag ? LASTO_ERR_TIMEOUT : LASTO_OK;
}

}  // namespace lasto
