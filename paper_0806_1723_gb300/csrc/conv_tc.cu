// 3x3x3 convolution of the learned-guess network on the fifth-generation tensor cores
// (tcgen05): an implicit GEMM, M = 128 nodes per CTA, N = cout, K = 27 taps x cin, issued as
// K = 16 steps (one tap, 16 input channels) of tcgen05.mma kind::f16 (BF16 x BF16 -> FP32)
// with the accumulator in tensor memory.
//
// A (128 x 16 per step) is gathered by the CTA's 128 threads, one node row each (the
// neighbour's 16 channels, zero outside the grid), into shared memory in the no-swizzle
// K-major core-matrix layout: 8 rows x 16 bytes per core matrix, the two K halves 128 bytes
// apart (leading byte offset), consecutive 8-row groups 256 bytes apart (stride byte
// offset).  B (cout x 16 per step) is stored in global memory already in that layout (packed
// once per weight set) and copied in.  Both arrive by cp.async (16-byte copies, zero-filled
// outside the grid) three steps ahead of their MMA, in a ring of five shared stages: one
// thread issues the MMA of a stage and commits it to the stage's mbarrier, which releases the
// stage for the copies of the step five later.  After the last step every thread reads its node's row of the
// accumulator (tcgen05.ld 32x32b: warp w owns tensor-memory lanes 32w .. 32w+31) and applies
// bias, ReLU and the output conversions.  Every mbarrier wait is bounded: on a timeout the
// kernel records an error, stops issuing, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace lasto {
namespace tc {

typedef __nv_bfloat16 bf16;

constexpr int TC_M = 128;        // nodes per CTA (MMA M), one per thread
constexpr int TC_STAGES = 5;
constexpr int TC_AHEAD = 3;      // steps whose operand copies are in flight
constexpr long long TC_SPIN_LIMIT = 1LL << 20;

struct Grid {
    int nb, D, H, W;
    __host__ __device__ size_t nodes() const { return (size_t)nb * D * H * W; }
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major, LBO 128 B, SBO 256 B, version 1
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(256 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M = 128, N
__host__ __device__ constexpr uint32_t make_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (long long it = 0; it < TC_SPIN_LIMIT; it++) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
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

// y = act(conv(x, w) + bias) for one 128-node tile; with part != null the raw sums of tap
// group blockIdx.y go to part[blockIdx.y][node][COUT] instead.
template <int COUT>
__global__ void __launch_bounds__(TC_M) k_conv_tc(Grid g, int cin, const bf16* __restrict__ x,
                                                 const uint4* __restrict__ wpk, const float* __restrict__ bias,
                                                 int relu, float* __restrict__ y32, int ldy32, int off32,
                                                 bf16* __restrict__ y16, int ldy16, int off16,
                                                 float* __restrict__ part, int* __restrict__ err)
{
    constexpr int A_BYTES = TC_M * 32;
    constexpr int B_BYTES = COUT * 32;
    constexpr int NCOL = COUT <= 32 ? 32 : (COUT <= 64 ? 64 : 128);
    __shared__ __align__(1024) unsigned char sA[TC_STAGES][A_BYTES];
    __shared__ __align__(1024) unsigned char sB[TC_STAGES][B_BYTES];
    __shared__ __align__(8) unsigned long long mbar[TC_STAGES];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const size_t N = g.nodes();
    const size_t node0 = (size_t)blockIdx.x * TC_M;

    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < TC_STAGES; s++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // this thread's node
    const size_t node = node0 + tid;
    const bool live = node < N;
    int b = 0, z = 0, yy = 0, xx = 0;
    if (live) {
        size_t r = node;
        xx = (int)(r % g.W);
        r /= g.W;
        yy = (int)(r % g.H);
        r /= g.H;
        z = (int)(r % g.D);
        b = (int)(r / g.D);
    }
    const int cpt = cin / 16;                       // K steps per tap
    const int tpg = 27 / gridDim.y, tap_a = blockIdx.y * tpg;
    const int nk = tpg * cpt;
    const uint32_t idesc = make_idesc(COUT);
    // canonical placement of this thread's row: 8-row group m8, row rr
    const int m8 = tid >> 3, rr = tid & 7;
    const int offA0 = (m8 * 2 + 0) * 128 + rr * 16, offA1 = (m8 * 2 + 1) * 128 + rr * 16;

    // issue the copies of step k into its stage (after the MMA that last read the stage)
    auto prefetch = [&](int k) {
        const int st = k % TC_STAGES;
        if (k >= TC_STAGES) {
            if (!mbar_wait(smem_u32(&mbar[st]), (uint32_t)((k / TC_STAGES - 1) & 1))) abort_flag = 1;
        }
        const int tap = tap_a + k / cpt, c0 = (k % cpt) * 16;
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        const int zz = z + dz, y2 = yy + dy, x2 = xx + dx;
        const bool in = live && zz >= 0 && zz < g.D && y2 >= 0 && y2 < g.H && x2 >= 0 && x2 < g.W;
        const size_t nbn = in ? (((size_t)b * g.D + zz) * g.H + y2) * g.W + x2 : 0;
        const bf16* src = x + nbn * cin + c0;
        const uint32_t n = in ? 16u : 0u;   // 0: the 16 bytes are zero-filled, nothing is read
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(&sA[st][offA0])), "l"(src),
                     "r"(n)
                     : "memory");
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(&sA[st][offA1])), "l"(src + 8),
                     "r"(n)
                     : "memory");
        const uint4* wsrc = wpk + ((size_t)(tap * cpt + c0 / 16)) * (B_BYTES / 16);
        for (int t = tid; t < B_BYTES / 16; t += TC_M)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(sB[st] + 16 * t)), "l"(wsrc + t)
                         : "memory");
    };
    for (int k = 0; k < TC_AHEAD; k++) {
        if (k < nk) prefetch(k);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    for (int kc = 0; kc < nk; kc++) {
        const int s = kc % TC_STAGES;
        if (kc + TC_AHEAD < nk) prefetch(kc + TC_AHEAD);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group %0;\n" ::"n"(TC_AHEAD) : "memory");   // step kc's copies have landed
        // make the shared-memory writes visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (abort_flag) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint64_t ad = make_desc(smem_u32(sA[s])), bd = make_desc(smem_u32(sB[s]));
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                    tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(kc > 0 ? 1 : 0)
                : "memory");
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&mbar[s]))
                         : "memory");
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    // wait for the last MMA (commits complete in issue order)
    if (!abort_flag && nk > 0) {
        const int s = (nk - 1) % TC_STAGES;
        if (!mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((nk - 1) / TC_STAGES) & 1))) abort_flag = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!abort_flag) {
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        float acc[COUT];
#pragma unroll
        for (int c = 0; c < COUT; c += 16) tmem_ld16(lane_base + (uint32_t)c, acc + c);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        // the accumulator rows leave through shared memory, 16 channels at a time, so that
        // consecutive threads store consecutive addresses (the A ring is idle now)
        float* stage = reinterpret_cast<float*>(&sA[0][0]);   // [TC_M][17]
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 16) {
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 16; j++) stage[tid * 17 + j] = acc[c0 + j];
            __syncthreads();
            for (int e = tid; e < TC_M * 16; e += TC_M) {
                const int r = e >> 4, j = e & 15, c = c0 + j;
                const size_t nd = node0 + r;
                if (nd >= N) continue;
                const float a = stage[r * 17 + j];
                if (part) {
                    part[((size_t)blockIdx.y * N + nd) * COUT + c] = a;
                } else {
                    float v = a + (bias ? bias[c] : 0.0f);
                    if (relu) v = fmaxf(v, 0.0f);
                    if (y32) y32[nd * ldy32 + off32 + c] = v;
                    if (y16) y16[nd * ldy16 + off16 + c] = __float2bfloat16(v);
                }
            }
        }
    } else if (tid == 0 && err) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOL) : "memory");
}

// Pack w [27][cin][cout] into the per-step B tiles: step k = tap * (cin/16) + c0/16 holds
// element (n = output channel, kk = input channel c0 + kk) at byte
// ((n/8)*2 + kk/8)*128 + (n%8)*16 + (kk%8)*2 of its cout*32-byte tile.
__global__ void k_pack_weights(int cin, int cout, const bf16* __restrict__ w, bf16* __restrict__ wpk)
{
    const size_t total = (size_t)27 * cin * cout;
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int co = (int)(t % cout);
    const int ci = (int)((t / cout) % cin);
    const int tap = (int)(t / ((size_t)cout * cin));
    const int step = tap * (cin / 16) + ci / 16, kk = ci % 16;
    const size_t byte = (size_t)step * cout * 32 + ((co / 8) * 2 + kk / 8) * 128 + (co % 8) * 16 + (kk % 8) * 2;
    wpk[byte / 2] = w[t];
}

__global__ void k_tc_epilogue(size_t N, int cout, int groups, const float* __restrict__ part,
                              const float* __restrict__ bias, int relu, float* __restrict__ y32, int ldy32, int off32,
                              bf16* __restrict__ y16, int ldy16, int off16)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= N * cout) return;
    const size_t nd = t / cout;
    const int co = (int)(t % cout);
    float v = part[t];
    for (int k = 1; k < groups; k++) v += part[(size_t)k * N * cout + t];
    v += bias ? bias[co] : 0.0f;
    if (relu) v = fmaxf(v, 0.0f);
    if (y32) y32[nd * ldy32 + off32 + co] = v;
    if (y16) y16[nd * ldy16 + off16 + co] = __float2bfloat16(v);
}

// ---------------------------------------------------------------- weight gradient
// dw[tap][ci][co] += sum over nodes of x[node + tap][ci] dy[node][co]: a GEMM with M = the
// (tap, ci) rows of a tile of taps (TPT = floor(128 / cin) taps, 128 rows, rows past TPT cin
// zero), N = cout, K = nodes, one CTA per (node chunk, tile).  Both operands are read
// MN-major from channels-last rows: a stage holds 64 nodes, for each node the TPT neighbour
// rows of cin channels (16-byte pieces; zero outside the grid) in A and its cout channels of
// dy in B, and is consumed by four K = 16 MMAs.  Core matrices (8 nodes x 8 channels, 128
// contiguous bytes) sit 128 bytes apart along the channels and 16 * rows bytes apart along
// the nodes; for these MN-major operands the descriptor's leading byte offset is the step
// along K (nodes) and its stride byte offset the step along M / N (channels) -- the other
// assignment reads outside the tiles (measured: wrong sums).  The accumulator (128 lanes x
// cout columns of tensor memory) is added to dw with FP32 atomics at the end.
constexpr int WG_STAGES = 3;
constexpr int WG_AHEAD = 2;
constexpr int WG_STEP = 64;                          // nodes per stage (four MMAs)
constexpr int WG_CHUNK = 2048;                       // nodes per CTA
constexpr int WG_A_BYTES = TC_M * 2 * WG_STEP;       // 128 rows x 64 nodes
__host__ __device__ constexpr int wg_smem(int cout) { return WG_STAGES * (WG_A_BYTES + cout * 2 * WG_STEP); }

__device__ __forceinline__ uint64_t make_desc_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(lbo >> 4) << 16;
    d |= (uint64_t)(sbo >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// node index -> (b, z, y, x) by multiply-high division by the invariant W, H, D (nodes < 2^31)
struct GridDiv {
    DivMagic w, h, d;
};

template <int COUT>
__global__ void __launch_bounds__(TC_M) k_conv_wgrad_tc(Grid g, GridDiv gd, int cin, const bf16* __restrict__ x,
                                                       const bf16* __restrict__ dy, float* __restrict__ dw,
                                                       int* __restrict__ err)
{
    constexpr int B_BYTES = COUT * 2 * WG_STEP;
    constexpr int NCOL = COUT <= 32 ? 32 : (COUT <= 64 ? 64 : 128);
    extern __shared__ __align__(1024) unsigned char wg_smem_raw[];
    unsigned char* sA = wg_smem_raw;                               // [WG_STAGES][WG_A_BYTES]
    unsigned char* sB = wg_smem_raw + WG_STAGES * WG_A_BYTES;      // [WG_STAGES][B_BYTES]
    __shared__ __align__(8) unsigned long long mbar[WG_STAGES];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const size_t N = g.nodes();
    const size_t node0 = (size_t)blockIdx.x * WG_CHUNK;
    const int tpt = TC_M / cin, tap0 = blockIdx.y * tpt;
    const int ntap = min(tpt, 27 - tap0);
    const int rows = ntap * cin;                                   // live rows of the tile
    const int r8n = rows / 8;                                      // 16-byte pieces per node in A

    // zero the ring (padding rows stay zero; no copy ever writes them)
    for (int t = tid; t < WG_STAGES * (WG_A_BYTES + B_BYTES) / 16; t += TC_M)
        reinterpret_cast<uint4*>(wg_smem_raw)[t] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        abort_flag = 0;
        for (int st = 0; st < WG_STAGES; st++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[st])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const size_t nodes = N > node0 ? min((size_t)WG_CHUNK, N - node0) : 0;
    const int nk = (int)((nodes + WG_STEP - 1) / WG_STEP);
    // core-matrix steps: along the channels (M / N) and along the nodes (K)
    constexpr uint32_t A_CH = 128, A_ND = 16 * 128, B_CH = 128, B_ND = (COUT / 8) * 128;
    const uint32_t idesc = make_idesc(COUT) | (1u << 15) | (1u << 16);   // A and B MN-major

    auto prefetch = [&](int k) {
        const int st = k % WG_STAGES;
        if (k >= WG_STAGES) {
            if (!mbar_wait(smem_u32(&mbar[st]), (uint32_t)((k / WG_STAGES - 1) & 1))) abort_flag = 1;
        }
        // A: piece p = (node kk, row group r8), r8 fastest (one node's row read contiguously)
        for (int p = tid; p < WG_STEP * r8n; p += TC_M) {
            const int kk = p / r8n, r8 = p - kk * r8n;
            const int m = r8 * 8, tl = m / cin, c0 = m - tl * cin;
            const size_t node = node0 + (size_t)k * WG_STEP + kk;
            bool in = node < N;
            size_t nbn = 0;
            if (in) {
                const unsigned r = (unsigned)node, q1 = div_by(r, gd.w), q2 = div_by(q1, gd.h), b = div_by(q2, gd.d);
                const int xx = (int)(r - q1 * (unsigned)g.W), yy = (int)(q1 - q2 * (unsigned)g.H);
                const int z = (int)(q2 - b * (unsigned)g.D);
                const int tap = tap0 + tl;
                const int zz = z + tap / 9 - 1, y2 = yy + (tap / 3) % 3 - 1, x2 = xx + tap % 3 - 1;
                in = zz >= 0 && zz < g.D && y2 >= 0 && y2 < g.H && x2 >= 0 && x2 < g.W;
                nbn = in ? (((size_t)b * g.D + zz) * g.H + y2) * g.W + x2 : 0;
            }
            const uint32_t dst = smem_u32(sA + st * WG_A_BYTES + r8 * A_CH + (kk >> 3) * A_ND + (kk & 7) * 16);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(x + nbn * cin + c0),
                         "r"(in ? 16u : 0u)
                         : "memory");
        }
        for (int p = tid; p < WG_STEP * (COUT / 8); p += TC_M) {
            const int kk = p / (COUT / 8), c8 = p - kk * (COUT / 8);
            const size_t node = node0 + (size_t)k * WG_STEP + kk;
            const bool in = node < N;
            const uint32_t dst = smem_u32(sB + st * B_BYTES + c8 * B_CH + (kk >> 3) * B_ND + (kk & 7) * 16);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst),
                         "l"(dy + (in ? node : 0) * COUT + c8 * 8), "r"(in ? 16u : 0u)
                         : "memory");
        }
    };
    for (int k = 0; k < WG_AHEAD; k++) {
        if (k < nk) prefetch(k);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    for (int kc = 0; kc < nk; kc++) {
        const int st = kc % WG_STAGES;
        if (kc + WG_AHEAD < nk) prefetch(kc + WG_AHEAD);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group %0;\n" ::"n"(WG_AHEAD) : "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (abort_flag) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int j = 0; j < WG_STEP / 16; j++) {   // 16 nodes = two core matrices along K
                const uint64_t ad = make_desc_mn(smem_u32(sA + st * WG_A_BYTES + j * 2 * A_ND), A_ND, A_CH);
                const uint64_t bd = make_desc_mn(smem_u32(sB + st * B_BYTES + j * 2 * B_ND), B_ND, B_CH);
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                        tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"((kc > 0 || j > 0) ? 1 : 0)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&mbar[st]))
                         : "memory");
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (!abort_flag && nk > 0) {
        const int st = (nk - 1) % WG_STAGES;
        if (!mbar_wait(smem_u32(&mbar[st]), (uint32_t)(((nk - 1) / WG_STAGES) & 1))) abort_flag = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!abort_flag && nk > 0) {
        // thread tid owns accumulator row m = tid (tensor-memory lane tid)
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        float acc[COUT];
#pragma unroll
        for (int c = 0; c < COUT; c += 16) tmem_ld16(lane_base + (uint32_t)c, acc + c);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        const int m = tid;
        if (m < rows) {
            const int tl = m / cin, ci = m - tl * cin;
            float* dst = dw + ((size_t)(tap0 + tl) * cin + ci) * COUT;
#pragma unroll
            for (int c = 0; c < COUT; c++) atomicAdd(dst + c, acc[c]);
        }
    } else if (abort_flag && tid == 0 && err) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOL) : "memory");
}

}  // namespace tc

cudaError_t launch_pack_weights(int cin, int cout, const void* w, void* wpk, cudaStream_t s)
{
    const size_t total = (size_t)27 * cin * cout;
    tc::k_pack_weights<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(cin, cout, (const tc::bf16*)w, (tc::bf16*)wpk);
    return cudaGetLastError();
}

int conv_fwd_tc(int nb, const int dims[3], int cin, int cout, const void* x, const void* wpk, const float* bias,
                int relu, float* y32, int ldy32, int off32, void* y16, int ldy16, int off16, float* scratch,
                size_t scratch_floats, int* err, void* stream)
{
    using namespace tc;
    if (nb < 1 || !dims || cin % 16 || cin < 16 || !x || !wpk ||
        !(cout == 16 || cout == 32 || cout == 48 || cout == 64 || cout == 96 || cout == 128))
        return LASTO_ERR_INVALID_ARG;
    Grid g{nb, dims[2], dims[1], dims[0]};
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned nbk = (unsigned)((g.nodes() + TC_M - 1) / TC_M);
    int groups = 1;
    if (scratch)
        for (int cand : {3, 9, 27})
            if ((size_t)nbk * cand <= 2432 && (size_t)cand * g.nodes() * cout <= scratch_floats) groups = cand;
    float* part = groups > 1 ? scratch : nullptr;
    const dim3 grid(nbk, groups);
    const bf16* X = (const bf16*)x;
    const uint4* W = (const uint4*)wpk;
    bf16* Y16 = (bf16*)y16;
#define LASTO_TC_CASE(C)                                                                                           \
    case C:                                                                                                        \
        k_conv_tc<C><<<grid, TC_M, 0, s>>>(g, cin, X, W, bias, relu, y32, ldy32, off32, Y16, ldy16, off16, part, err); \
        break;
    switch (cout) {
        LASTO_TC_CASE(16)
        LASTO_TC_CASE(32)
        LASTO_TC_CASE(48)
        LASTO_TC_CASE(64)
        LASTO_TC_CASE(96)
        LASTO_TC_CASE(128)
        default: return LASTO_ERR_INVALID_ARG;
    }
#undef LASTO_TC_CASE
    if (part) {
        const size_t n = g.nodes() * cout;
        k_tc_epilogue<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g.nodes(), cout, groups, part, bias, relu, y32,
                                                                  ldy32, off32, Y16, ldy16, off16);
    }
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

int conv_wgrad_tc(int nb, const int dims[3], int cin, int cout, const void* x, const void* dy16, float* dw,
                  int* err, void* stream)
{
    using namespace tc;
    if (nb < 1 || !dims || cin % 16 || cin < 16 || cin > 128 || !x || !dy16 || !dw ||
        !(cout == 16 || cout == 32 || cout == 48 || cout == 64 || cout == 96 || cout == 128))
        return LASTO_ERR_INVALID_ARG;
    Grid g{nb, dims[2], dims[1], dims[0]};
    if (g.nodes() == 0) return LASTO_OK;
    if (g.nodes() >= (size_t(1) << 31)) return LASTO_ERR_INVALID_ARG;
    const GridDiv gd{div_magic((unsigned)g.W), div_magic((unsigned)g.H), div_magic((unsigned)g.D)};
    cudaStream_t s = (cudaStream_t)stream;
    const int tpt = TC_M / cin;
    const dim3 grid((unsigned)((g.nodes() + WG_CHUNK - 1) / WG_CHUNK), (unsigned)((27 + tpt - 1) / tpt));
    const bf16* X = (const bf16*)x;
    const bf16* DY = (const bf16*)dy16;
#define LASTO_WG_CASE(C)                                                                                 \
    case C:                                                                                              \
        if (cudaFuncSetAttribute(k_conv_wgrad_tc<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, wg_smem(C)) != \
            cudaSuccess)                                                                                 \
            return LASTO_ERR_CUDA;                                                                       \
        k_conv_wgrad_tc<C><<<grid, TC_M, wg_smem(C), s>>>(g, gd, cin, X, DY, dw, err);                     \
        break;
    switch (cout) {
        LASTO_WG_CASE(16)
        LASTO_WG_CASE(32)
        LASTO_WG_CASE(48)
        LASTO_WG_CASE(64)
        LASTO_WG_CASE(96)
        LASTO_WG_CASE(128)
        default: return LASTO_ERR_INVALID_ARG;
    }
#undef LASTO_WG_CASE
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

}  // namespace lasto
