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

#include <cuda_fp16.h>

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

// The 56 monomial terms of the real solid harmonics r^l y_lm (l <= 4) as (index, lm, a, b, c)
// of x^a y^b z^c, in the order of the library's monomial table (checked against it at setup);
// the coefficients come from that table.
#define HS_TERMS(X)                                                                                              \
    X(0, 0, 0, 0, 0) X(1, 1, 0, 1, 0) X(2, 2, 0, 0, 1) X(3, 3, 1, 0, 0) X(4, 4, 1, 1, 0) X(5, 5, 0, 1, 1)        \
    X(6, 6, 0, 0, 2) X(7, 6, 2, 0, 0) X(8, 6, 0, 2, 0) X(9, 7, 1, 0, 1) X(10, 8, 2, 0, 0) X(11, 8, 0, 2, 0)      \
    X(12, 9, 2, 1, 0) X(13, 9, 0, 3, 0) X(14, 10, 1, 1, 1) X(15, 11, 0, 1, 2) X(16, 11, 2, 1, 0)                 \
    X(17, 11, 0, 3, 0) X(18, 12, 0, 0, 3) X(19, 12, 2, 0, 1) X(20, 12, 0, 2, 1) X(21, 13, 1, 0, 2)               \
    X(22, 13, 3, 0, 0) X(23, 13, 1, 2, 0) X(24, 14, 2, 0, 1) X(25, 14, 0, 2, 1) X(26, 15, 3, 0, 0)               \
    X(27, 15, 1, 2, 0) X(28, 16, 3, 1, 0) X(29, 16, 1, 3, 0) X(30, 17, 2, 1, 1) X(31, 17, 0, 3, 1)               \
    X(32, 18, 1, 1, 2) X(33, 18, 3, 1, 0) X(34, 18, 1, 3, 0) X(35, 19, 0, 1, 3) X(36, 19, 2, 1, 1)               \
    X(37, 19, 0, 3, 1) X(38, 20, 0, 0, 4) X(39, 20, 4, 0, 0) X(40, 20, 0, 4, 0) X(41, 20, 2, 2, 0)               \
    X(42, 20, 2, 0, 2) X(43, 20, 0, 2, 2) X(44, 21, 1, 0, 3) X(45, 21, 3, 0, 1) X(46, 21, 1, 2, 1)               \
    X(47, 22, 2, 0, 2) X(48, 22, 0, 2, 2) X(49, 22, 4, 0, 0) X(50, 22, 0, 4, 0) X(51, 23, 3, 0, 1)               \
    X(52, 23, 1, 2, 1) X(53, 24, 4, 0, 0) X(54, 24, 2, 2, 0) X(55, 24, 0, 4, 0)
constexpr int HS_L3_TERMS = 28;   // terms of l <= 3 (the l = 4 terms follow)

__constant__ float c_hs_coef[N_MONO_TERMS];

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
    bool same = true;
#define HS_CHECK(i, LM, EA, EB, EC) same = same && t[i].lm == LM && t[i].a == EA && t[i].b == EB && t[i].c == EC;
    HS_TERMS(HS_CHECK)
#undef HS_CHECK
    if (!same) return cudaErrorInvalidValue;
    float coef[N_MONO_TERMS];
    for (int i = 0; i < N_MONO_TERMS; i++) coef[i] = (float)t[i].coef;
    e = cudaMemcpyToSymbol(c_hs_coef, coef, sizeof(coef));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_hs_mono, o.data(), sizeof(MonoF32) * o.size());
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_hs_first, first, sizeof(first));
    if (e == cudaSuccess) g_hs_device = dev;
    return e;
}

struct HsBasis {
    int per;                        // functions per atom
    int nb, lmax;
    int n[HS_MAXB], l[HS_MAXB], off[HS_MAXB];   // off: first function of the entry within its atom
    float zeta[HS_MAXB];
    unsigned char q_of[HS_MAXF];    // function within an atom -> table entry
    signed char m_of[HS_MAXF];      // -> m
};

struct HsGrid {
    int nx, ny, nz, na;
    const double *x, *y, *z, *pos, *R;
};

// Inside a sphere: |P - pos_a| < R_a in FP64; an FP32 pass settles every atom whose squared
// distance is not within 0.1 % of R_a^2 (FP32 rounding of the coordinates moves it by < 1e-5).
__device__ __forceinline__ bool hs_inside(const HsGrid& g, const float4* __restrict__ at4, int i, int j, int k)
{
    const float px = (float)g.x[i], py = (float)g.y[j], pz = (float)g.z[k];
    for (int a = 0; a < g.na; a++) {
        const float4 A = __ldg(at4 + a);
        const float ex = px - A.x, ey = py - A.y, ez = pz - A.z;
        const float d2f = ex * ex + ey * ey + ez * ez;
        if (d2f < 0.999f * A.w) return true;
        if (d2f <= 1.001f * A.w) {
            const double dx = g.x[i] - g.pos[3 * a], dy = g.y[j] - g.pos[3 * a + 1], dz = g.z[k] - g.pos[3 * a + 2];
            const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            if (sqrt(d2) < g.R[a]) return true;
        }
    }
    return false;
}

// FP32 copies of the spheres for the prefilter: (x, y, z, R^2)
__global__ void k_hs_atoms(int na, const double* __restrict__ pos, const double* __restrict__ R, float4* __restrict__ at4)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < na) at4[a] = make_float4((float)pos[3 * a], (float)pos[3 * a + 1], (float)pos[3 * a + 2], (float)(R[a] * R[a]));
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
__global__ void __launch_bounds__(256) k_hs_count(HsGrid g, const float4* __restrict__ at4, int* __restrict__ cnt)
{
    __shared__ int wt[8];
    const size_t N = (size_t)g.nx * g.ny * g.nz;
    int c = 0;
    for (int e = 0; e < HS_CNT / 256; e++) {
        const size_t P = (size_t)blockIdx.x * HS_CNT + e * 256 + threadIdx.x;
        if (P < N) {
            const int i = (int)(P % g.nx), j = (int)((P / g.nx) % g.ny), k = (int)(P / ((size_t)g.nx * g.ny));
            c += !hs_inside(g, at4, i, j, k);
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
__global__ void __launch_bounds__(256) k_hs_scatter(HsGrid g, const float4* __restrict__ at4, const int* __restrict__ off,
                                                    int* __restrict__ idx, float* __restrict__ sw)
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
            f = !hs_inside(g, at4, i, j, k);
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

// (2', 3') The contraction on the fifth-generation tensor cores.  Every table value x (A or
// T, scaled by a power of two per function so that |x| < 2^14) is split into two FP16 parts,
// x_hi = fp16(x) and x_lo = fp16(x - x_hi), 22 significant bits together (the splitting error
// stays below 2^-25 absolute in scaled units, far under FP32 rounding of the sums); a product
// is taken as hi*hi + hi*lo + lo*hi (the dropped lo*lo is below 2^-22 of it), exact in the FP32
// accumulator.  So S takes 3 tcgen05.mma kind::f16 (M = N = 128, K = 16 nodes) per 16 nodes
// and 2H = A_I T_J^T + T_I A_J^T takes 6, into two 128-column tensor-memory regions.
//
// The table kernel writes the operands already in the MMA's shared-memory layout (no-swizzle
// K-major core matrices of 8 rows x 16 bytes; the two 8-node halves of a K step 128 bytes
// apart, 8-function groups 256 bytes apart): one 4 KiB image per (16 nodes, 128 functions,
// array), the four arrays (A_hi, A_lo, T_hi, T_lo) of a block adjacent, so that a stage of a
// tile is two 16 KiB bulk copies (cp.async.bulk, completion counted on an mbarrier).
//
// Warp roles (10 warps): one thread issues the bulk copies into a ring of six 32 KiB stages,
// one thread issues the MMAs (and frees a stage by tcgen05.commit to its mbarrier) into the
// accumulators (tensor-memory columns 0-127 S, 128-255 2H; lane = function row), and eight
// warps (warp w: lanes 32 (w % 4) .. +31, S for w < 4 and 2H for w >= 4) add each HS_IV-node
// interval's sums into the unit's FP32 partial sums, which stay in tensor memory (columns
// 256-511; tcgen05.ld, add, tcgen05.st), so that no FP32 accumulation inside the tensor core
// is longer than one interval.  A work unit is one upper-triangle tile and HS_SEG nodes,
// numbered segment-major so that the CTAs running together read the same table rows (from
// L2); at a unit's end the drain warps form its partial sums in FP64, undo the scales
// (exponent arithmetic) and add them to S and 2H by FP64 atomic addition while the MMAs run on.
constexpr int TC_TM = 128;                       // functions per tile side (MMA M and N)
constexpr int TC_NT = 320;                       // threads: 8 drain warps, producer, MMA issuer
constexpr int TC_SK = 16;                        // nodes per stage (one MMA K step)
constexpr int TC_IMG = TC_TM * TC_SK * 2;        // one FP16 operand image: 4 KiB
constexpr int TC_SIDE = 4 * TC_IMG;              // A_hi, A_lo, T_hi, T_lo of one function block
constexpr int TC_STAGE = 2 * TC_SIDE;            // the I and J blocks of a tile
constexpr int TC_RING = 6;
constexpr int TC_SMEM = TC_RING * TC_STAGE + 128;
constexpr int HS_IV = 512;                       // nodes per FP32 accumulation interval
constexpr int HS_SEG = 2048;                     // nodes per work unit
constexpr int HS_SCALE_MAX = 14;                 // scaled |x| < 2^14

__device__ __forceinline__ uint32_t hs_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t hs_now()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: false after about two seconds or once *abort is set
// (then *abort is set).
__device__ __forceinline__ bool hs_wait(uint32_t mbar, uint32_t parity, volatile int* abort)
{
    uint64_t t0 = 0;
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (*abort) return false;
        const uint64_t t = hs_now();
        if (t0 == 0) {
            t0 = t;
        } else if (t - t0 > 2000000000ull) {
            *abort = 1;
            return false;
        }
    }
}

__device__ __forceinline__ uint64_t hs_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;   // leading byte offset: the second 8-node half
    d |= (uint64_t)(256 >> 4) << 32;   // stride byte offset: the next 8-function group
    d |= (uint64_t)1 << 46;
    return d;
}

// FP32 accumulator, FP16 A and B, both K-major, M = N = 128
constexpr uint32_t HS_IDESC = (1u << 4) | ((uint32_t)(TC_TM >> 3) << 17) | ((uint32_t)(TC_TM >> 4) << 24);

__device__ __forceinline__ void hs_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(HS_IDESC), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void hs_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
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

// phi and phi~ (FP32, times sqrt(Vol)) of every function of atom `at` at listed node P:
// out(loc, phi, phi~) for loc in [0, per).  The 25 solid harmonics first (straight-line, the
// same monomial terms in every lane), then per table entry its radial factors and its 2l+1
// functions (a switch on l keeps the harmonic index a compile-time constant).
template <typename Out>
__device__ __forceinline__ void hs_eval_atom(const HsBasis& B, const HsGrid& g, int P, float w, float Vp, int at,
                                             Out&& out)
{
    const int i = P % g.nx, j = (P / g.nx) % g.ny, k = P / (g.nx * g.ny);
    const float dx = (float)(g.x[i] - g.pos[3 * at]), dy = (float)(g.y[j] - g.pos[3 * at + 1]),
                dz = (float)(g.z[k] - g.pos[3 * at + 2]);
    const float r = sqrtf(dx * dx + dy * dy + dz * dz);
    const float ir = 1.0f / r;
    float px[5], py[5], pz[5];
    px[0] = py[0] = pz[0] = 1.0f;
#pragma unroll
    for (int e = 1; e < 5; e++) {
        px[e] = px[e - 1] * dx;
        py[e] = py[e - 1] * dy;
        pz[e] = pz[e - 1] * dz;
    }
    float sh[NLM];
#pragma unroll
    for (int lm = 0; lm < NLM; lm++) sh[lm] = 0.0f;
#define HS_ACC(i, LM, EA, EB, EC) \
    if (i < HS_L3_TERMS || B.lmax >= 4) sh[LM] = fmaf(c_hs_coef[i], px[EA] * py[EB] * pz[EC], sh[LM]);
    HS_TERMS(HS_ACC)
#undef HS_ACC
#pragma unroll 1
    for (int q = 0; q < B.nb; q++) {
        const int n = B.n[q], l = B.l[q], f0 = B.off[q];
        const float zt = B.zeta[q];
        float rad = w * expf(-zt * r);
        for (int t = 0; t < n - 1 - l; t++) rad *= r;   // sqrt(Vol) r^(n-1-l) e^{-zeta r}
        const float fac =
            0.5f * ((float)(l * (l + 1) - n * (n - 1)) * ir * ir + 2.0f * zt * (float)n * ir - zt * zt) + Vp;
#define HS_OUT(m, LM)                         \
    {                                         \
        const float ph = rad * sh[LM];        \
        out(f0 + (m), ph, fac * ph);          \
    }
        switch (l) {
        case 0: HS_OUT(0, 0) break;
        case 1: HS_OUT(0, 1) HS_OUT(1, 2) HS_OUT(2, 3) break;
        case 2: HS_OUT(0, 4) HS_OUT(1, 5) HS_OUT(2, 6) HS_OUT(3, 7) HS_OUT(4, 8) break;
        case 3: HS_OUT(0, 9) HS_OUT(1, 10) HS_OUT(2, 11) HS_OUT(3, 12) HS_OUT(4, 13) HS_OUT(5, 14) HS_OUT(6, 15) break;
        default:
            HS_OUT(0, 16) HS_OUT(1, 17) HS_OUT(2, 18) HS_OUT(3, 19) HS_OUT(4, 20) HS_OUT(5, 21) HS_OUT(6, 22)
            HS_OUT(7, 23) HS_OUT(8, 24) break;
        }
#undef HS_OUT
    }
}

__device__ __forceinline__ float hs_warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// (2'a) scale exponents from closed-form bounds over the interstitial nodes (r >= R_a from
// the function's own atom): |phi_f| <= sqrt(max Vol) max_{r >= R_a} r^(n-1) e^{-zeta r}
// sqrt(2 (2l+1) / 4pi) (real harmonics) and |phi~_f| <= (|kinetic factor at R_a, terms in
// absolute value| + max |V| over the listed nodes) times that.  e_f makes the first bound
// < 2^14; one c makes every second bound times 2^(e_f + c) < 2^14.  ea[f] = e_f, ea[M] = c.
// One block.
__device__ __forceinline__ int hs_scale_exp(float bound, int lo, int hi)
{
    int x = 0;
    if (!(bound > 0.0f)) return 0;
    frexpf(bound, &x);
    return min(hi, max(lo, HS_SCALE_MAX - x));
}

// max |V| over the listed nodes (non-negative floats as ordered integers)
__global__ void __launch_bounds__(256) k_hs_vmax(const int* __restrict__ idx, int n_list, const double* __restrict__ V,
                                                 unsigned* __restrict__ vmax)
{
    float m = 0.0f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_list; p += gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf((float)V[idx[p]]));
    m = hs_warp_max(m);
    if ((threadIdx.x & 31) == 0) atomicMax(vmax, __float_as_uint(m));
}

__global__ void __launch_bounds__(1024) k_hs_bounds(HsBasis B, HsGrid g, const unsigned* __restrict__ vmax,
                                                    int* __restrict__ ea)
{
    __shared__ float red[32];
    __shared__ float s_w, s_v;
    auto block_max = [&](float v) {
        v = hs_warp_max(v);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        float r = 0.0f;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) r = fmaxf(r, red[q]);
        return r;
    };
    // largest dual-cell volume and |V| over the listed nodes
    float w = 1.0f;
    const double* ax[3] = {g.x, g.y, g.z};
    const int nn[3] = {g.nx, g.ny, g.nz};
    for (int d = 0; d < 3; d++) {
        float m = 0.0f;
        for (int q = threadIdx.x; q < nn[d]; q += blockDim.x) m = fmaxf(m, (float)hs_dual(ax[d], nn[d], q));
        w *= block_max(m);
    }
    const float vm = __uint_as_float(*vmax);
    if (threadIdx.x == 0) {
        s_w = sqrtf(w) * 1.001f;
        s_v = vm * 1.001f;
    }
    __syncthreads();
    const int M = g.na * B.per;
    float rt = 0.0f;
    for (int f = threadIdx.x; f < M; f += blockDim.x) {
        const int at = f / B.per, q = B.q_of[f - at * B.per];
        const int n = B.n[q], l = B.l[q];
        const float zt = B.zeta[q], Ra = (float)g.R[at];
        const float rs = fmaxf(Ra, (float)(n - 1) / zt);   // the radial factor peaks at (n-1)/zeta
        float rad = expf(-zt * rs);
        for (int t = 0; t < n - 1; t++) rad *= rs;
        const float bphi = 1.01f * s_w * rad * sqrtf(2.0f * (2 * l + 1) / (4.0f * 3.14159265f));
        const float kin = 0.5f * (fabsf((float)(l * (l + 1) - n * (n - 1))) / (Ra * Ra) + 2.0f * zt * n / Ra + zt * zt);
        const int e = hs_scale_exp(bphi, -100, 100);
        ea[f] = e;
        rt = fmaxf(rt, ldexpf((kin + s_v) * bphi, e));
    }
    rt = block_max(rt);
    if (threadIdx.x == 0) ea[M] = hs_scale_exp(rt, -20, 20);
}

// (2'c) the FP16 operand images of one chunk: rows p in [0, K) are listed nodes p0 + p (zero
// past n_list); functions past M keep the zeros the tables were cleared to.  Block: 32 nodes
// (lanes) x 8 atoms (warps).  Each warp stages its atom's four FP16 arrays for its 32 nodes in
// shared memory ([array][function][node]) and writes them out as 16-byte pieces (8 nodes of one
// function), so that a warp store fills whole 128-byte lines (8 consecutive functions).
__global__ void __launch_bounds__(256) k_hs_basis16(const __grid_constant__ HsBasis B, HsGrid g, int nT, const int* __restrict__ idx,
                                                    const float* __restrict__ sw, const double* __restrict__ V,
                                                    const int* __restrict__ ea, int p0, int n_list,
                                                    __half* __restrict__ img)
{
    extern __shared__ __align__(16) __half hs_stage[];   // [8 warps][4][per][32]
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, at = blockIdx.y * 8 + wp;
    if (at >= g.na) return;
    __half* st = hs_stage + (size_t)wp * 4 * B.per * 32;
    const int p = blockIdx.x * 32 + lane;   // row within the chunk
    const bool live = p0 + p < n_list;
    const int P = live ? idx[p0 + p] : 0;
    const int ec = ea[g.na * B.per];
    hs_eval_atom(B, g, P, live ? sw[p0 + p] : 0.0f, live ? (float)V[P] : 0.0f, at, [&](int loc, float ph, float pt) {
        const int e = ea[at * B.per + loc];
        const float a = live ? ph * __int_as_float((127 + e) << 23) : 0.0f;
        const float t = live ? pt * __int_as_float((127 + e + ec) << 23) : 0.0f;
        const __half ah = __float2half_rn(a), th = __float2half_rn(t);
        st[(0 * B.per + loc) * 32 + lane] = ah;
        st[(1 * B.per + loc) * 32 + lane] = __float2half_rn(a - __half2float(ah));
        st[(2 * B.per + loc) * 32 + lane] = th;
        st[(3 * B.per + loc) * 32 + lane] = __float2half_rn(t - __half2float(th));
    });
    __syncwarp();
    // piece (array, function, kb, k half): 8 nodes = 16 bytes
    const int kb0 = blockIdx.x * 2;
    for (int t = lane; t < 4 * B.per * 4; t += 32) {
        const int arr = t / (4 * B.per), rem = t - arr * 4 * B.per, loc = rem >> 2, kbh = rem & 3;
        const int kb = kb0 + (kbh >> 1), kh = kbh & 1;
        const int f = at * B.per + loc, fb = f >> 7, r = f & 127;
        const uint4 v = *reinterpret_cast<const uint4*>(st + (arr * B.per + loc) * 32 + (kbh >> 1) * 16 + kh * 8);
        __half* dst = img + ((size_t)kb * nT + fb) * (TC_SIDE / 2) + arr * (TC_IMG / 2) + (r >> 3) * 128 + kh * 64 +
                      (r & 7) * 8;
        *reinterpret_cast<uint4*>(dst) = v;
    }
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

__device__ __forceinline__ void hs_tmem_st16(uint32_t taddr, const float* v)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};\n" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
        "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
        "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}

// x * 2^-e for a double x whose result stays a normal number: the exponent field lowered by e
__device__ __forceinline__ double hs_unscale(float v, int e)
{
    const double x = (double)v;
    return v == 0.0f ? 0.0 : __longlong_as_double(__double_as_longlong(x) - ((long long)e << 52));
}

__global__ void __launch_bounds__(TC_NT, 1) k_hs_gemm_tc(int M, int nT, const unsigned char* __restrict__ img, int K,
                                                        int units, const int* __restrict__ ea,
                                                        double* __restrict__ S, double* __restrict__ H2,
                                                        int* __restrict__ err)
{
    extern __shared__ unsigned char hs_dyn[];
    unsigned char* ring = reinterpret_cast<unsigned char*>(((uintptr_t)hs_dyn + 127) & ~(uintptr_t)127);
    __shared__ __align__(8) unsigned long long full[TC_RING], empty[TC_RING], accf, acce;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int pairs = nT * (nT + 1) / 2;

    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < TC_RING; s++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(hs_smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(hs_smem_u32(&empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(hs_smem_u32(&accf)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 256;\n" ::"r"(hs_smem_u32(&acce)) : "memory");
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
    int last_mma = -1;   // the MMA thread's last committed stage

    if (warp == 8 && lane == 0) {
        // ---------------- producer: two bulk copies per stage
        int g = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
            const HsUnit w = hs_unit(u, pairs, nT, K);
            for (int r0 = w.k0; r0 < w.k1 && ok; r0 += TC_SK, g++) {
                const int slot = g % TC_RING;
                if (g >= TC_RING && !hs_wait(hs_smem_u32(&empty[slot]), (uint32_t)((g / TC_RING - 1) & 1), &abort_flag)) {
                    ok = false;
                    break;
                }
                const uint32_t fb = hs_smem_u32(&full[slot]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(TC_STAGE)
                             : "memory");
                const size_t kb = (size_t)(r0 / TC_SK) * nT;
                const unsigned char* srcI = img + (kb + w.I) * TC_SIDE;
                const unsigned char* srcJ = img + (kb + w.J) * TC_SIDE;
                const uint32_t dst = hs_smem_u32(ring + (size_t)slot * TC_STAGE);
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                        dst),
                    "l"(srcI), "r"(TC_SIDE), "r"(fb)
                    : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                        dst + TC_SIDE),
                    "l"(srcJ), "r"(TC_SIDE), "r"(fb)
                    : "memory");
            }
        }
        if (!ok) {
            // copies still in flight land before the CTA leaves
            for (int q = max(0, g - TC_RING); q < g; q++) {
                volatile int never = 0;
                hs_wait(hs_smem_u32(&full[q % TC_RING]), (uint32_t)((q / TC_RING) & 1), &never);
            }
        }
    } else if (warp == 9 && lane == 0) {
        // ---------------- MMA issuer: accumulators in columns 0-127 (S) and 128-255 (2H)
        int g = 0, ic = 0;
        bool ok = true;
        const uint32_t tS = tmem, tH = tmem + TC_TM;
        for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
            const HsUnit w = hs_unit(u, pairs, nT, K);
            for (int c0 = w.k0; c0 < w.k1 && ok; c0 += HS_IV, ic++) {
                const int c1 = min(w.k1, c0 + HS_IV);
                // the previous interval has been drained
                if (ic >= 1 && !hs_wait(hs_smem_u32(&acce), (uint32_t)((ic - 1) & 1), &abort_flag)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                for (int r0 = c0; r0 < c1; r0 += TC_SK, g++) {
                    const int slot = g % TC_RING;
                    if (!hs_wait(hs_smem_u32(&full[slot]), (uint32_t)((g / TC_RING) & 1), &abort_flag)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t sb = hs_smem_u32(ring + (size_t)slot * TC_STAGE);
                    const uint64_t aIh = hs_desc(sb), aIl = hs_desc(sb + TC_IMG);
                    const uint64_t tIh = hs_desc(sb + 2 * TC_IMG), tIl = hs_desc(sb + 3 * TC_IMG);
                    const uint64_t aJh = hs_desc(sb + TC_SIDE), aJl = hs_desc(sb + TC_SIDE + TC_IMG);
                    const uint64_t tJh = hs_desc(sb + TC_SIDE + 2 * TC_IMG), tJl = hs_desc(sb + TC_SIDE + 3 * TC_IMG);
                    const uint32_t acc = r0 > c0 ? 1u : 0u;
                    hs_mma(tS, aIh, aJh, acc);
                    hs_mma(tS, aIh, aJl, 1u);
                    hs_mma(tS, aIl, aJh, 1u);
                    hs_mma(tH, aIh, tJh, acc);
                    hs_mma(tH, aIh, tJl, 1u);
                    hs_mma(tH, aIl, tJh, 1u);
                    hs_mma(tH, tIh, aJh, 1u);
                    hs_mma(tH, tIh, aJl, 1u);
                    hs_mma(tH, tIl, aJh, 1u);
                    hs_commit(hs_smem_u32(&empty[slot]));
                    last_mma = g;
                }
                if (ok) hs_commit(hs_smem_u32(&accf));
            }
        }
    } else if (warp < 8) {
        // ---------------- drain: row = tensor-memory lane; S (warps 0-3) or 2H (4-7) columns of
        // the interval added into the unit's partial sums 256 columns further on
        const int q = warp & 3, half = warp >> 2, row = 32 * q + lane;
        const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(half * TC_TM);
        const uint32_t tp = ta + 2 * TC_TM;
        int ic = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
            const HsUnit w = hs_unit(u, pairs, nT, K);
            for (int c0 = w.k0; c0 < w.k1; c0 += HS_IV, ic++) {
                const bool got = hs_wait(hs_smem_u32(&accf), (uint32_t)(ic & 1), &abort_flag);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    abort_flag = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const bool first = c0 == w.k0;
#pragma unroll 1
                for (int cc = 0; cc < TC_TM; cc += 32) {
                    float v[32], pv[32];
                    hs_tmem_ld16(ta + (uint32_t)cc, v);
                    hs_tmem_ld16(ta + (uint32_t)(cc + 16), v + 16);
                    if (!first) {
                        hs_tmem_ld16(tp + (uint32_t)cc, pv);
                        hs_tmem_ld16(tp + (uint32_t)(cc + 16), pv + 16);
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    if (!first)
#pragma unroll
                        for (int jj = 0; jj < 32; jj++) v[jj] += pv[jj];
                    hs_tmem_st16(tp + (uint32_t)cc, v);
                    hs_tmem_st16(tp + (uint32_t)(cc + 16), v + 16);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(hs_smem_u32(&acce)) : "memory");
            }
            if (!ok) break;
            // the unit's sums: FP64, scales undone, into S or 2H
            const int a = w.I * TC_TM + row;
            const int e_a = a < M ? ea[a] + (half ? ea[M] : 0) : 0;
            double* dst = (half ? H2 : S) + (size_t)(a < M ? a : 0) * M;
#pragma unroll 1
            for (int cc = 0; cc < TC_TM; cc += 16) {
                float v[16];
                hs_tmem_ld16(tp + (uint32_t)cc, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (a >= M) continue;
#pragma unroll
                for (int jj = 0; jj < 16; jj++) {
                    const int b = w.J * TC_TM + cc + jj;
                    if (b < M && a <= b) atomicAdd(dst + b, hs_unscale(v[jj], e_a + __ldg(ea + b)));
                }
            }
        }
    }
    __syncthreads();
    if (abort_flag) {
        // the MMAs already issued finish before the tensor memory is released
        if (warp == 9 && lane == 0 && last_mma >= 0) {
            volatile int never = 0;
            hs_wait(hs_smem_u32(&empty[last_mma % TC_RING]), (uint32_t)((last_mma / TC_RING) & 1), &never);
        }
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
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_hs_basis16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(8 * 4 * HS_MAXF * 32 * sizeof(__half)));
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

size_t hs_scratch_bytes(const int n[3], int M, int na)
{
    const size_t N = (size_t)n[0] * n[1] * n[2];
    const size_t nblk = (N + HS_CNT - 1) / HS_CNT;
    const int Mp = (M + TC_TM - 1) / TC_TM * TC_TM;   // the larger padding of the two contractions
    const size_t K = hs_rows_per_chunk(N, Mp);
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    return up(sizeof(int) * nblk) + up(sizeof(int) * (nblk + 1)) + up(sizeof(int) * N) + up(sizeof(float) * N) +
           up(8 * (size_t)Mp * K) +
           up(sizeof(int) * (Mp + 1)) + 2 * up(sizeof(int)) + up(sizeof(float) * 4 * na);
}

// scratch: hs_scratch_bytes(n, M) bytes, 256-byte aligned; carved into the block counts,
// offsets, listed nodes, sqrt(Vol), the basis tables (FP32 A and T for the SIMT contraction,
// FP16 operand images for the tensor cores), the per-function scale exponents, an error flag
// and the FP32 copies of the spheres.  Synchronises the stream twice
// (the number of listed nodes sizes the chunk loop; the error flag is read at the end).
int launch_interstitial_hs(const int n[3], const double* x, const double* y, const double* z, int na,
                           const double* pos, const double* R, int nb, const int* bn, const int* bl,
                           const double* bz, const double* V, double* S, double* H, void* scratch, int mode,
                           lasto_hs_stats* stats, cudaStream_t s)
{
    int per = 0;
    if (hs_basis_check(nb, bn, bl, bz, &per) != LASTO_OK) return LASTO_ERR_INVALID_ARG;
    if (mode < LASTO_HS_DEFAULT || mode > LASTO_HS_TENSOR) return LASTO_ERR_INVALID_ARG;
    const bool tensor = mode != LASTO_HS_SIMT;
    HsBasis B{};
    B.per = per;
    B.nb = nb;
    for (int q = 0, f = 0; q < nb; q++) {
        B.n[q] = bn[q];
        B.l[q] = bl[q];
        B.off[q] = f;
        B.zeta[q] = (float)bz[q];
        B.lmax = std::max(B.lmax, bl[q]);
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
    const int Mp128 = (M + TC_TM - 1) / TC_TM * TC_TM;
    const size_t Kmax = hs_rows_per_chunk(N, Mp128);
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
    char* tables = carve(8 * (size_t)Mp128 * Kmax);
    float* A = reinterpret_cast<float*>(tables);                  // SIMT: [K][Mp] FP32 each
    float* T = A + (size_t)Mp * Kmax;
    int* ea = reinterpret_cast<int*>(carve(sizeof(int) * (Mp128 + 1)));
    int* err = reinterpret_cast<int*>(carve(sizeof(int)));
    unsigned* vmax = reinterpret_cast<unsigned*>(carve(sizeof(unsigned)));
    float4* at4 = reinterpret_cast<float4*>(carve(sizeof(float4) * na));

    const HsGrid g{n[0], n[1], n[2], na, x, y, z, pos, R};
    // optional device timing: events around the list, every chunk's two kernels and the mirror
    std::vector<cudaEvent_t> ev;
    auto mark = [&]() {
        if (!stats) return;
        cudaEvent_t t;
        if (cudaEventCreate(&t) == cudaSuccess) {
            cudaEventRecord(t, s);
            ev.push_back(t);
        }
    };
    struct EvFree {
        std::vector<cudaEvent_t>& v;
        ~EvFree()
        {
            for (cudaEvent_t t : v) cudaEventDestroy(t);
        }
    } ev_free{ev};
    cudaError_t e = cudaMemsetAsync(S, 0, sizeof(double) * (size_t)M * M, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(H, 0, sizeof(double) * (size_t)M * M, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e != cudaSuccess) return LASTO_ERR_CUDA;
    mark();
    k_hs_atoms<<<(na + 127) / 128, 128, 0, s>>>(na, pos, R, at4);
    k_hs_count<<<nblk, 256, 0, s>>>(g, at4, cnt);
    k_hs_scan<<<1, 1024, 0, s>>>(nblk, cnt, off);
    k_hs_scatter<<<nblk, 256, 0, s>>>(g, at4, off, idx, sw);
    mark();
    int n_list = 0;
    e = cudaMemcpyAsync(&n_list, off + nblk, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return LASTO_ERR_CUDA;

    const unsigned ablocks = (unsigned)((na + 7) / 8);
    if (tensor && n_list > 0) {
        // per-function scales; operand images cleared once (the padding functions past M stay zero)
        e = cudaMemsetAsync(tables, 0, 8 * (size_t)Mp128 * Kmax, s);
        if (e != cudaSuccess) return LASTO_ERR_CUDA;
        e = cudaMemsetAsync(vmax, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return LASTO_ERR_CUDA;
        k_hs_vmax<<<(unsigned)std::min(4 * sms, (n_list + 255) / 256), 256, 0, s>>>(idx, n_list, V, vmax);
        k_hs_bounds<<<1, 1024, 0, s>>>(B, g, vmax, ea);
    }
    const int pairs = nT * (nT + 1) / 2;
    for (int p0 = 0; p0 < n_list; p0 += (int)Kmax) {
        const int K = (int)std::min<size_t>(Kmax, ((size_t)(n_list - p0) + HS_KC - 1) / HS_KC * HS_KC);
        mark();
        if (tensor) {
            k_hs_basis16<<<dim3((unsigned)(K / 32), ablocks), 256, (size_t)8 * 4 * per * 32 * sizeof(__half), s>>>(
                B, g, nT, idx, sw, V, ea, p0, n_list, reinterpret_cast<__half*>(tables));
        } else {
            const size_t tot = (size_t)K * Mp;
            const unsigned gb = (unsigned)std::min<size_t>((tot + 255) / 256, (size_t)sms * 16);
            k_hs_basis<<<gb, 256, 0, s>>>(B, g, M, Mp, idx, sw, V, p0, n_list, K, A, T);
        }
        mark();
        if (tensor) {
            const int units = pairs * ((K + HS_SEG - 1) / HS_SEG);
            const int grid = std::min(units, sms);
            k_hs_gemm_tc<<<grid, TC_NT, TC_SMEM, s>>>(M, nT, reinterpret_cast<const unsigned char*>(tables), K, units,
                                                       ea, S, H, err);
        } else {
            // node ranges per tile: about eight CTAs per SM in all
            int split = std::max(1, (8 * sms + pairs - 1) / pairs);
            split = std::min(split, K / HS_KC);
            const int kper = (K / HS_KC + split - 1) / split * HS_KC;
            split = (K + kper - 1) / kper;
            k_hs_gemm_f32<<<dim3((unsigned)pairs, (unsigned)split), HS_NT, 0, s>>>(M, Mp, nT, A, T, kper, K, S, H);
        }
        mark();
    }
    mark();
    k_hs_mirror<<<(unsigned)(((size_t)M * M + 255) / 256), 256, 0, s>>>(M, S, H);
    mark();
    if (cudaGetLastError() != cudaSuccess) return LASTO_ERR_CUDA;
    int flag = 0;
    e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return LASTO_ERR_CUDA;
    if (stats) {
        const int chunks = n_list > 0 ? (int)((n_list + Kmax - 1) / Kmax) : 0;
        *stats = lasto_hs_stats{};
        stats->interstitial_nodes = n_list;
        stats->chunks = chunks;
        stats->tile = tile;
        auto span = [&](size_t i, size_t j) {
            float ms = 0.0f;
            if (j < ev.size() && cudaEventElapsedTime(&ms, ev[i], ev[j]) != cudaSuccess) ms = 0.0f;
            return ms;
        };
        if (ev.size() == (size_t)(2 + 3 * chunks + 2)) {
            stats->ms_list = span(0, 1);
            for (int c = 0; c < chunks; c++) {
                stats->ms_tables += span(2 + 3 * c, 3 + 3 * c);
                stats->ms_contract += span(3 + 3 * c, 4 + 3 * c);
            }
            stats->ms_mirror = span(2 + 3 * chunks, 3 + 3 * chunks);
        }
    }
    return flag ? LASTO_ERR_TIMEOUT : LASTO_OK;
}

}  // namespace lasto
