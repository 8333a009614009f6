// Kernels of the small 3-D U-Net that predicts the coarse-grid potential used as the
// multigrid initial guess (BF16 tensor-core convolutions accumulating in FP32).
//
// Layout: activations are channels-last, [node][channel] with node = ((b*D + z)*H + y)*W + x
// over a batch of D x H x W node grids; convolution weights are [27 taps][cin][cout] with
// tap = (dz*3 + dy)*3 + dx for offsets -1..1, zero padding, stride 1.  cin and cout are
// multiples of 16.  A convolution is an implicit GEMM: M = nodes, N = cout, K = 27 cin, run
// on warp-level BF16 tensor-core MMA (16x16x16 fragments) with FP32 accumulators.
// Down- and up-sampling act on the node index grid (n -> (n+1)/2 and back): full-weighting
// average (boundary planes renormalised) and trilinear interpolation, with exact adjoints.
#include <cuda_bf16.h>
#include <mma.h>

#include "internal.cuh"

namespace lasto {
namespace nn {

using namespace nvcuda;
typedef __nv_bfloat16 bf16;

constexpr int CT = 128;     // threads per convolution block (4 warps)
constexpr int CM = 64;      // output nodes per block

struct Grid {
    int nb, D, H, W;
    __host__ __device__ size_t nodes() const { return (size_t)nb * D * H * W; }
};

__device__ __forceinline__ void split(size_t node, const Grid& g, int& b, int& z, int& y, int& x)
{
    x = (int)(node % g.W);
    size_t r = node / g.W;
    y = (int)(r % g.H);
    r /= g.H;
    z = (int)(r % g.D);
    b = (int)(r / g.D);
}

// y = act(conv(x, w) + bias); act = relu if relu != 0.  Writes FP32 (ldy32, off32) and / or
// BF16 (ldy16, off16) outputs, either may be null.  With part != null the block sums only the
// taps of its group blockIdx.y (27 / gridDim.y taps) and stores the raw sums to
// part[blockIdx.y][node][COUT]; k_conv_epilogue then adds the groups in order.
template <int COUT>
__global__ void __launch_bounds__(CT) k_conv_fwd(Grid g, int cin, const bf16* __restrict__ x,
                                                 const bf16* __restrict__ w, const float* __restrict__ bias, int relu,
                                                 float* __restrict__ y32, int ldy32, int off32, bf16* __restrict__ y16,
                                                 int ldy16, int off16, float* __restrict__ part)
{
    __shared__ __align__(32) bf16 As[CM * 16];
    __shared__ __align__(32) bf16 Bs[16 * COUT];
    __shared__ __align__(32) float Cs[CM * COUT];
    const int warp = threadIdx.x >> 5;
    const size_t node0 = (size_t)blockIdx.x * CM;
    const size_t N = g.nodes();
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[COUT / 16];
#pragma unroll
    for (int n = 0; n < COUT / 16; n++) wmma::fill_fragment(acc[n], 0.0f);
    // each thread stages 8 channels of one row of A
    const int row = threadIdx.x >> 1, half = threadIdx.x & 1;
    const size_t node = node0 + row;
    int b = 0, z = 0, yy = 0, xx = 0;
    const bool live = node < N;
    if (live) split(node, g, b, z, yy, xx);
    const int tpg = 27 / gridDim.y, tap_a = blockIdx.y * tpg;
    for (int tap = tap_a; tap < tap_a + tpg; tap++) {
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        const int zz = z + dz, y2 = yy + dy, x2 = xx + dx;
        const bool in = live && zz >= 0 && zz < g.D && y2 >= 0 && y2 < g.H && x2 >= 0 && x2 < g.W;
        const size_t nb_node = in ? (((size_t)b * g.D + zz) * g.H + y2) * g.W + x2 : 0;
        for (int c0 = 0; c0 < cin; c0 += 16) {
            uint4 v = make_uint4(0, 0, 0, 0);
            if (in) v = *reinterpret_cast<const uint4*>(x + nb_node * cin + c0 + half * 8);
            *reinterpret_cast<uint4*>(As + row * 16 + half * 8) = v;
            const bf16* wt = w + ((size_t)tap * cin + c0) * COUT;
            for (int t = threadIdx.x; t < 16 * COUT / 8; t += CT)
                reinterpret_cast<uint4*>(Bs)[t] = reinterpret_cast<const uint4*>(wt)[t];
            __syncthreads();
            wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> af;
            wmma::load_matrix_sync(af, As + warp * 16 * 16, 16);
#pragma unroll
            for (int n = 0; n < COUT / 16; n++) {
                wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> bfm;
                wmma::load_matrix_sync(bfm, Bs + n * 16, COUT);
                wmma::mma_sync(acc[n], af, bfm, acc[n]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int n = 0; n < COUT / 16; n++)
        wmma::store_matrix_sync(Cs + warp * 16 * COUT + n * 16, acc[n], COUT, wmma::mem_row_major);
    __syncthreads();
    if (part) {
        float* dst = part + ((size_t)blockIdx.y * N + node0) * COUT;
        for (int t = threadIdx.x; t < CM * COUT; t += CT)
            if (node0 + t / COUT < N) dst[t] = Cs[t];
        return;
    }
    for (int t = threadIdx.x; t < CM * COUT; t += CT) {
        const int r = t / COUT, co = t % COUT;
        const size_t nd = node0 + r;
        if (nd >= N) continue;
        float v = Cs[t] + (bias ? bias[co] : 0.0f);
        if (relu) v = fmaxf(v, 0.0f);
        if (y32) y32[nd * ldy32 + off32 + co] = v;
        if (y16) y16[nd * ldy16 + off16 + co] = __float2bfloat16(v);
    }
}

// sum of the tap groups (in group order), bias, activation, outputs
__global__ void k_conv_epilogue(size_t N, int cout, int groups, const float* __restrict__ part,
                                const float* __restrict__ bias, int relu, float* __restrict__ y32, int ldy32,
                                int off32, bf16* __restrict__ y16, int ldy16, int off16)
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

// dw[tap][ci][co] += sum_node x[node + tap][ci] dy[node][co];  dbias[co] += sum_node dy[node][co]
// (block: one tap, 16 input channels, a chunk of nodes; FP32 atomics into dw).
constexpr int WCH = 1024;   // nodes per wgrad block
template <int COUT>
__global__ void __launch_bounds__(CT) k_conv_wgrad(Grid g, int cin, const bf16* __restrict__ x,
                                                   const bf16* __restrict__ dy, float* __restrict__ dw)
{
    __shared__ __align__(32) bf16 At[4][16 * 16];
    __shared__ __align__(32) bf16 Bt[4][16 * COUT];
    __shared__ __align__(32) float Cs[4][16 * COUT];
    const int tap = blockIdx.y, c0 = blockIdx.z * 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int dz = tap / 9 - 1, dyo = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const size_t N = g.nodes();
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[COUT / 16];
#pragma unroll
    for (int n = 0; n < COUT / 16; n++) wmma::fill_fragment(acc[n], 0.0f);
    const size_t chunk0 = (size_t)blockIdx.x * WCH;
    for (size_t s0 = chunk0 + (size_t)warp * 16; s0 < chunk0 + WCH && s0 < N; s0 += 4 * 16) {
        // A^T tile: 16 nodes x 16 channels of x at the shifted node (lane: node lane/2, half lane%2)
        {
            const int r = lane >> 1, half = lane & 1;
            const size_t node = s0 + r;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (node < N) {
                int b, z, yy, xx;
                split(node, g, b, z, yy, xx);
                const int zz = z + dz, y2 = yy + dyo, x2 = xx + dx;
                if (zz >= 0 && zz < g.D && y2 >= 0 && y2 < g.H && x2 >= 0 && x2 < g.W) {
                    const size_t nn = (((size_t)b * g.D + zz) * g.H + y2) * g.W + x2;
                    v = *reinterpret_cast<const uint4*>(x + nn * cin + c0 + half * 8);
                }
            }
            *reinterpret_cast<uint4*>(At[warp] + r * 16 + half * 8) = v;
            // dy rows of the 16 nodes
            for (int t = lane; t < 16 * COUT / 8; t += 32) {
                const int rr = t / (COUT / 8), cc = t % (COUT / 8);
                const size_t nd = s0 + rr;
                uint4 q = make_uint4(0, 0, 0, 0);
                if (nd < N) q = reinterpret_cast<const uint4*>(dy + nd * COUT)[cc];
                reinterpret_cast<uint4*>(Bt[warp])[t] = q;
            }
        }
        __syncwarp();
        wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> af;   // (ci, node) = At[node][ci]
        wmma::load_matrix_sync(af, At[warp], 16);
#pragma unroll
        for (int n = 0; n < COUT / 16; n++) {
            wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> bfm;
            wmma::load_matrix_sync(bfm, Bt[warp] + n * 16, COUT);
            wmma::mma_sync(acc[n], af, bfm, acc[n]);
        }
        __syncwarp();
    }
#pragma unroll
    for (int n = 0; n < COUT / 16; n++)
        wmma::store_matrix_sync(Cs[warp] + n * 16, acc[n], COUT, wmma::mem_row_major);
    __syncthreads();
    for (int t = threadIdx.x; t < 16 * COUT; t += CT) {
        const float v = Cs[0][t] + Cs[1][t] + Cs[2][t] + Cs[3][t];
        const int ci = t / COUT, co = t % COUT;
        atomicAdd(dw + ((size_t)tap * cin + c0 + ci) * COUT + co, v);
    }
}

// dbias[co] += sum over nodes of dy[node][co] (FP32 gradient): each block sums a span of node
// rows with the threads along the row (coalesced), reduces per channel in shared memory and
// adds its partial with one atomic per channel
constexpr int BG_ROWS = 128;    // node rows per block
__global__ void __launch_bounds__(256) k_bias_grad(size_t N, int cout, const float* __restrict__ dy,
                                                   float* __restrict__ db)
{
    __shared__ float sm[256];
    const int per = 256 / cout;                      // rows in flight per block step
    const int t = threadIdx.x, c = t % cout, r0 = t / cout;
    float acc = 0.0f;
    if (r0 < per) {
        const size_t first = (size_t)blockIdx.x * BG_ROWS, last = min(first + BG_ROWS, N);
        for (size_t n = first + r0; n < last; n += per) acc += dy[n * cout + c];
    }
    sm[t] = acc;
    __syncthreads();
    if (t < cout) {
        float s = 0.0f;
        for (int r = 0; r < per; r++) s += sm[r * cout + t];
        atomicAdd(db + t, s);
    }
}

// w_t[tap'][co][ci] = w[26 - tap'][ci][co]: the weights of the data-gradient convolution
__global__ void k_flip_weights(int cin, int cout, const bf16* __restrict__ w, bf16* __restrict__ wt)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t total = (size_t)27 * cin * cout;
    if (t >= total) return;
    const int ci = (int)(t % cin);
    const size_t r = t / cin;
    const int co = (int)(r % cout), tp = (int)(r / cout);
    wt[t] = w[((size_t)(26 - tp) * cin + ci) * cout + co];
}

// ---------------------------------------------------------------- elementwise
__global__ void k_relu_grad(size_t n, const float* __restrict__ y, const float* __restrict__ dy, float* __restrict__ dx,
                            bf16* __restrict__ dx16)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float v = y[t] > 0.0f ? dy[t] : 0.0f;
    if (dx) dx[t] = v;
    if (dx16) dx16[t] = __float2bfloat16(v);
}

__global__ void k_to_bf16(size_t n, const float* __restrict__ a, bf16* __restrict__ b)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t < n) b[t] = __float2bfloat16(a[t]);
}

// dst[node][doff + c] (+)= src[node][soff + c], c < C
__global__ void k_copy_channels(size_t nodes, int C, const float* __restrict__ src, int lds, int soff,
                                float* __restrict__ dst, int ldd, int doff, int accumulate)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= nodes * C) return;
    const size_t n = t / C;
    const int c = (int)(t % C);
    const float v = src[n * lds + soff + c];
    float* d = dst + n * ldd + doff + c;
    *d = accumulate ? *d + v : v;
}

// full-weighting average onto the every-other-node grid (boundary planes renormalised)
__device__ __forceinline__ float fw_w(int a, int I, int nc)
{
    // weights of offsets a = -1, 0, 1 around coarse node I, renormalised at the two ends
    if (I == 0) return a < 0 ? 0.0f : (a == 0 ? 2.0f / 3.0f : 1.0f / 3.0f);
    if (I == nc - 1) return a > 0 ? 0.0f : (a == 0 ? 2.0f / 3.0f : 1.0f / 3.0f);
    return a == 0 ? 0.5f : 0.25f;
}

__global__ void k_down(Grid gf, Grid gc, int C, const float* __restrict__ x, float* __restrict__ y)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= gc.nodes() * C) return;
    const int c = (int)(t % C);
    int b, Z, Y, X;
    split(t / C, gc, b, Z, Y, X);
    float acc = 0.0f;
    for (int a = -1; a <= 1; a++) {
        const float wz = fw_w(a, Z, gc.D);
        if (wz == 0.0f) continue;
        for (int bb = -1; bb <= 1; bb++) {
            const float wy = fw_w(bb, Y, gc.H);
            if (wy == 0.0f) continue;
            for (int cc = -1; cc <= 1; cc++) {
                const float wx = fw_w(cc, X, gc.W);
                if (wx == 0.0f) continue;
                const size_t f = (((size_t)b * gf.D + 2 * Z + a) * gf.H + 2 * Y + bb) * gf.W + 2 * X + cc;
                acc = fmaf(wz * wy * wx, x[f * C + c], acc);
            }
        }
    }
    y[t] = acc;
}

// adjoint of k_down: dx[fine] = sum over coarse nodes that use it of weight * dy[coarse]
__global__ void k_down_adj(Grid gf, Grid gc, int C, const float* __restrict__ dy, float* __restrict__ dx)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= gf.nodes() * C) return;
    const int c = (int)(t % C);
    int b, z, y, x;
    split(t / C, gf, b, z, y, x);
    float acc = 0.0f;
    for (int Z = (z - 1) / 2; Z <= (z + 1) / 2; Z++) {
        const int a = z - 2 * Z;
        if (Z < 0 || Z >= gc.D || a < -1 || a > 1) continue;
        const float wz = fw_w(a, Z, gc.D);
        for (int Y = (y - 1) / 2; Y <= (y + 1) / 2; Y++) {
            const int bb = y - 2 * Y;
            if (Y < 0 || Y >= gc.H || bb < -1 || bb > 1) continue;
            const float wy = fw_w(bb, Y, gc.H);
            for (int X = (x - 1) / 2; X <= (x + 1) / 2; X++) {
                const int cc = x - 2 * X;
                if (X < 0 || X >= gc.W || cc < -1 || cc > 1) continue;
                const float wx = fw_w(cc, X, gc.W);
                const size_t q = (((size_t)b * gc.D + Z) * gc.H + Y) * gc.W + X;
                acc = fmaf(wz * wy * wx, dy[q * C + c], acc);
            }
        }
    }
    dx[t] = acc;
}

// trilinear interpolation of the coarse node grid at the fine nodes; writes channels
// [off, off + C) of a row of stride ldy
__global__ void k_up(Grid gf, Grid gc, int C, const float* __restrict__ x, float* __restrict__ y, int ldy, int off)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= gf.nodes() * C) return;
    const int c = (int)(t % C);
    int b, z, yy, xx;
    split(t / C, gf, b, z, yy, xx);
    float acc = 0.0f;
    const int z0 = z >> 1, y0 = yy >> 1, x0 = xx >> 1;
    const int nz = (z & 1) ? 2 : 1, ny = (yy & 1) ? 2 : 1, nx = (xx & 1) ? 2 : 1;
    const float wz = nz == 2 ? 0.5f : 1.0f, wy = ny == 2 ? 0.5f : 1.0f, wx = nx == 2 ? 0.5f : 1.0f;
    for (int a = 0; a < nz; a++)
        for (int bb = 0; bb < ny; bb++)
            for (int cc = 0; cc < nx; cc++) {
                const size_t q = (((size_t)b * gc.D + z0 + a) * gc.H + y0 + bb) * gc.W + x0 + cc;
                acc = fmaf(wz * wy * wx, x[q * C + c], acc);
            }
    y[(t / C) * ldy + off + c] = acc;
}

// adjoint of k_up: dx[coarse] = sum over fine nodes f near 2I of weight * dy[f] (channels [off, off+C))
__global__ void k_up_adj(Grid gf, Grid gc, int C, const float* __restrict__ dy, int ldy, int off, float* __restrict__ dx)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= gc.nodes() * C) return;
    const int c = (int)(t % C);
    int b, Z, Y, X;
    split(t / C, gc, b, Z, Y, X);
    float acc = 0.0f;
    for (int a = -1; a <= 1; a++) {
        const int z = 2 * Z + a;
        if (z < 0 || z >= gf.D) continue;
        const float wz = a == 0 ? 1.0f : 0.5f;
        for (int bb = -1; bb <= 1; bb++) {
            const int y = 2 * Y + bb;
            if (y < 0 || y >= gf.H) continue;
            const float wy = bb == 0 ? 1.0f : 0.5f;
            for (int cc = -1; cc <= 1; cc++) {
                const int x = 2 * X + cc;
                if (x < 0 || x >= gf.W) continue;
                const float wx = cc == 0 ? 1.0f : 0.5f;
                const size_t f = (((size_t)b * gf.D + z) * gf.H + y) * gf.W + x;
                acc = fmaf(wz * wy * wx, dy[f * ldy + off + c], acc);
            }
        }
    }
    dx[t] = acc;
}

// loss = sum mask (p - t)^2 / count;  dp = 2 mask (p - t) / count.  One block per 1024 nodes,
// FP64 atomics for the loss (reporting only).
__global__ void k_mse(size_t n, const float* __restrict__ p, const float* __restrict__ tgt, const float* __restrict__ mask,
                      float inv_count, float* __restrict__ dp, double* __restrict__ loss)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (t < n) {
        const float d = (p[t] - tgt[t]) * (mask ? mask[t] : 1.0f);
        dp[t] = 2.0f * d * inv_count;
        l = d * d * inv_count;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, (double)l);
}

// Adam (Kingma & Ba 2015) on FP32 master weights; also writes the BF16 copy
__global__ void k_adam(size_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                       bf16* __restrict__ w16)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.0f - b1) * gt;
    const float vt = b2 * v[t] + (1.0f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    const float wt = w[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
    w[t] = wt;
    if (w16) w16[t] = __float2bfloat16(wt);
}

// Network input at the coarse nodes: channel 0 = b h^2 * s0 (the source in grid units),
// channel 1 = Dirichlet face value * s1 (0 inside), channel 2 = log(h / h_ref) with h the
// local dual-cell size (dual_x dual_y dual_z)^(1/3); channels 3..15 = 0.
__global__ void k_guess_features(int nx, int ny, int nz, const double* __restrict__ b, const double* __restrict__ faces,
                                 const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
                                 float s0, float s1, float h_ref, float* __restrict__ out)
{
    const size_t N = (size_t)nx * ny * nz;
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= N) return;
    const int i = (int)(t % nx), j = (int)((t / nx) % ny), k = (int)(t / ((size_t)nx * ny));
    auto dual = [](const double* c, int n, int q) {
        return q == 0 ? 0.5 * (c[1] - c[0]) : q == n - 1 ? 0.5 * (c[n - 1] - c[n - 2]) : 0.5 * (c[q + 1] - c[q - 1]);
    };
    const double h = cbrt(dual(x, nx, i) * dual(y, ny, j) * dual(z, nz, k));
    const bool face = i == 0 || j == 0 || k == 0 || i == nx - 1 || j == ny - 1 || k == nz - 1;
    float* o = out + t * 16;
    o[0] = face ? 0.0f : (float)(b[t] * h * h) * s0;
    o[1] = face ? (float)faces[t] * s1 : 0.0f;
    o[2] = (float)log(h / h_ref);
    for (int c = 3; c < 16; c++) o[c] = 0.0f;
}

// coarse-grid guess: interior = prediction / s, faces = the Dirichlet values
__global__ void k_guess_grid(size_t N, int nx, int ny, int nz, const float* __restrict__ pred, int ld, float inv_s,
                             const double* __restrict__ faces, double* __restrict__ u)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= N) return;
    const int i = (int)(t % nx), j = (int)((t / nx) % ny), k = (int)(t / ((size_t)nx * ny));
    const bool face = i == 0 || j == 0 || k == 0 || i == nx - 1 || j == ny - 1 || k == nz - 1;
    u[t] = face ? faces[t] : (double)(pred[t * ld] * inv_s);
}

inline unsigned blocks(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace nn
}  // namespace lasto

namespace lasto {

// Convolution launcher.  Small grids leave most SMs idle with one block per 64 nodes, so
// when scratch is given the 27 taps are split into 3, 9 or 27 groups (the largest split
// that keeps the grid within 2432 blocks, 16 per SM) summed by k_conv_epilogue.
int conv_fwd(int nb, const int dims[3], int cin, int cout, const void* x, const void* w, const float* bias, int relu,
             float* y32, int ldy32, int off32, void* y16, int ldy16, int off16, float* scratch,
             size_t scratch_floats, void* stream)
{
    using namespace nn;
    if (nb < 1 || !dims || cin % 16 || cout % 16 || cin < 16 || cout < 16 || cout > 128 || !x || !w)
        return LASTO_ERR_INVALID_ARG;
    Grid g{nb, dims[2], dims[1], dims[0]};
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned nbk = blocks(g.nodes(), CM);
    int groups = 1;
    if (scratch)
        for (int cand : {3, 9, 27})
            if ((size_t)nbk * cand <= 2432 && (size_t)cand * nbk * CM * cout <= scratch_floats) groups = cand;
    float* part = groups > 1 ? scratch : nullptr;
    const dim3 grid(nbk, groups);
    const bf16* X = (const bf16*)x;
    const bf16* Wt = (const bf16*)w;
    bf16* Y16 = (bf16*)y16;
    switch (cout) {
        case 16: k_conv_fwd<16><<<grid, CT, 0, s>>>(g, cin, X, Wt, bias, relu, y32, ldy32, off32, Y16, ldy16, off16, part); break;
        case 32: k_conv_fwd<32><<<grid, CT, 0, s>>>(g, cin, X, Wt, bias, relu, y32, ldy32, off32, Y16, ldy16, off16, part); break;
        case 48: k_conv_fwd<48><<<grid, CT, 0, s>>>(g, cin, X, Wt, bias, relu, y32, ldy32, off32, Y16, ldy16, off16, part); break;
        case 64: k_conv_fwd<64><<<grid, CT, 0, s>>>(g, cin, X, Wt, bias, relu, y32, ldy32, off32, Y16, ldy16, off16, part); break;
        case 96: k_conv_fwd<96><<<grid, CT, 0, s>>>(g, cin, X, Wt, bias, relu, y32, ldy32, off32, Y16, ldy16, off16, part); break;
        case 128: k_conv_fwd<128><<<grid, CT, 0, s>>>(g, cin, X, Wt, bias, relu, y32, ldy32, off32, Y16, ldy16, off16, part); break;
        default: return LASTO_ERR_INVALID_ARG;
    }
    if (part) {
        const size_t n = g.nodes() * cout;
        k_conv_epilogue<<<blocks(n, 256), 256, 0, s>>>(g.nodes(), cout, groups, part, bias, relu, y32, ldy32, off32,
                                                       Y16, ldy16, off16);
    }
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

}  // namespace lasto

using namespace lasto::nn;

extern "C" {

int lasto_nn_conv3d_fwd(int nb, const int dims[3], int cin, int cout, const void* x, const void* w, const float* bias,
                        int relu, float* y32, int ldy32, int off32, void* y16, int ldy16, int off16, void* stream)
{
    return lasto::conv_fwd(nb, dims, cin, cout, x, w, bias, relu, y32, ldy32, off32, y16, ldy16, off16, nullptr, 0,
                           stream);
}

int lasto_nn_pack_weights(int cin, int cout, const void* w, void* wpk, void* stream)
{
    if (cin < 16 || cin % 16 || cout < 16 || cout % 16 || !w || !wpk) return LASTO_ERR_INVALID_ARG;
    return lasto::launch_pack_weights(cin, cout, w, wpk, (cudaStream_t)stream) == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

int lasto_nn_conv3d_fwd_tc(int nb, const int dims[3], int cin, int cout, const void* x, const void* wpk,
                           const float* bias, int relu, float* y32, int ldy32, int off32, void* y16, int ldy16,
                           int off16, int* err, void* stream)
{
    return lasto::conv_fwd_tc(nb, dims, cin, cout, x, wpk, bias, relu, y32, ldy32, off32, y16, ldy16, off16, nullptr,
                              0, err, stream);
}

int lasto_nn_conv3d_dgrad(int nb, const int dims[3], int cin, int cout, const void* dy, const void* w, void* w_flip,
                          float* dx32, void* stream)
{
    if (!w_flip || !dx32) return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nw = (size_t)27 * cin * cout;
    k_flip_weights<<<blocks(nw, 256), 256, 0, s>>>(cin, cout, (const bf16*)w, (bf16*)w_flip);
    if (cudaGetLastError() != cudaSuccess) return LASTO_ERR_CUDA;
    return lasto_nn_conv3d_fwd(nb, dims, cout, cin, dy, w_flip, nullptr, 0, dx32, cin, 0, nullptr, 0, 0, stream);
}

int lasto_nn_conv3d_wgrad(int nb, const int dims[3], int cin, int cout, const void* x, const void* dy16,
                          const float* dy32, float* dw, float* db, void* stream)
{
    if (nb < 1 || !dims || cin % 16 || cout % 16 || cout > 128 || !x || !dy16 || !dw) return LASTO_ERR_INVALID_ARG;
    Grid g{nb, dims[2], dims[1], dims[0]};
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 grid(blocks(g.nodes(), WCH), 27, cin / 16);
    const bf16* X = (const bf16*)x;
    const bf16* DY = (const bf16*)dy16;
    switch (cout) {
        case 16: k_conv_wgrad<16><<<grid, CT, 0, s>>>(g, cin, X, DY, dw); break;
        case 32: k_conv_wgrad<32><<<grid, CT, 0, s>>>(g, cin, X, DY, dw); break;
        case 48: k_conv_wgrad<48><<<grid, CT, 0, s>>>(g, cin, X, DY, dw); break;
        case 64: k_conv_wgrad<64><<<grid, CT, 0, s>>>(g, cin, X, DY, dw); break;
        default: return LASTO_ERR_INVALID_ARG;
    }
    if (db && dy32) k_bias_grad<<<blocks(g.nodes(), BG_ROWS), 256, 0, s>>>(g.nodes(), cout, dy32, db);
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

int lasto_nn_conv3d_dgrad_tc(int nb, const int dims[3], int cin, int cout, const void* dy, const void* w, void* w_flip,
                             void* wpk_flip, float* dx32, int* err, void* stream)
{
    if (!w || !w_flip || !wpk_flip || !dx32 || cin < 16 || cin % 16 || cout < 16 || cout % 16) return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nw = (size_t)27 * cin * cout;
    k_flip_weights<<<blocks(nw, 256), 256, 0, s>>>(cin, cout, (const bf16*)w, (bf16*)w_flip);
    if (cudaGetLastError() != cudaSuccess) return LASTO_ERR_CUDA;
    // the data gradient is the forward convolution of dy with the flipped, transposed weights
    if (lasto::launch_pack_weights(cout, cin, w_flip, wpk_flip, s) != cudaSuccess) return LASTO_ERR_CUDA;
    return lasto::conv_fwd_tc(nb, dims, cout, cin, dy, wpk_flip, nullptr, 0, dx32, cin, 0, nullptr, 0, 0, nullptr, 0,
                              err, stream);
}

int lasto_nn_conv3d_wgrad_tc(int nb, const int dims[3], int cin, int cout, const void* x, const void* dy16,
                             const float* dy32, float* dw, float* db, int* err, void* stream)
{
    if (nb < 1 || !dims || !x || !dy16 || !dw) return LASTO_ERR_INVALID_ARG;
    const int st = lasto::conv_wgrad_tc(nb, dims, cin, cout, x, dy16, dw, err, stream);
    if (st) return st;
    if (db && dy32) {
        Grid g{nb, dims[2], dims[1], dims[0]};
        k_bias_grad<<<blocks(g.nodes(), BG_ROWS), 256, 0, (cudaStream_t)stream>>>(g.nodes(), cout, dy32, db);
    }
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

int lasto_nn_relu_grad(size_t n, const float* y, const float* dy, float* dx, void* dx16, void* stream)
{
    k_relu_grad<<<blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(n, y, dy, dx, (bf16*)dx16);
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

int lasto_nn_to_bf16(size_t n, const float* a, void* b, void* stream)
{
    k_to_bf16<<<blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(n, a, (bf16*)b);
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

int lasto_nn_copy_channels(size_t nodes, int C, const float* src, int lds, int soff, float* dst, int ldd, int doff,
                           int accumulate, void* stream)
{
    k_copy_channels<<<blocks(nodes * C, 256), 256, 0, (cudaStream_t)stream>>>(nodes, C, src, lds, soff, dst, ldd, doff,
                                                                              accumulate);
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

int lasto_nn_down(int nb, const int fine[3], int C, const float* x, float* y, int adjoint, void* stream)
{
    if (nb < 1 || !fine || fine[0] % 2 == 0 || fine[1] % 2 == 0 || fine[2] % 2 == 0) return LASTO_ERR_INVALID_ARG;
    Grid gf{nb, fine[2], fine[1], fine[0]};
    Grid gc{nb, (fine[2] + 1) / 2, (fine[1] + 1) / 2, (fine[0] + 1) / 2};
    cudaStream_t s = (cudaStream_t)stream;
    if (!adjoint) k_down<<<blocks(gc.nodes() * C, 256), 256, 0, s>>>(gf, gc, C, x, y);
    else k_down_adj<<<blocks(gf.nodes() * C, 256), 256, 0, s>>>(gf, gc, C, x, y);
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

int lasto_nn_up(int nb, const int fine[3], int C, const float* x, float* y, int ldy, int off, int adjoint, void* stream)
{
    if (nb < 1 || !fine || fine[0] % 2 == 0 || fine[1] % 2 == 0 || fine[2] % 2 == 0) return LASTO_ERR_INVALID_ARG;
    Grid gf{nb, fine[2], fine[1], fine[0]};
    Grid gc{nb, (fine[2] + 1) / 2, (fine[1] + 1) / 2, (fine[0] + 1) / 2};
    cudaStream_t s = (cudaStream_t)stream;
    if (!adjoint) k_up<<<blocks(gf.nodes() * C, 256), 256, 0, s>>>(gf, gc, C, x, y, ldy, off);
    else k_up_adj<<<blocks(gc.nodes() * C, 256), 256, 0, s>>>(gf, gc, C, x, ldy, off, y);
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

int lasto_nn_mse(size_t n, const float* p, const float* t, const float* mask, float inv_count, float* dp, double* loss,
                 void* stream)
{
    k_mse<<<blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(n, p, t, mask, inv_count, dp, loss);
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

int lasto_nn_guess_features(const int n[3], const double* b, const double* faces, const double* x, const double* y,
                            const double* z, float s0, float s1, float h_ref, float* out, void* stream)
{
    if (!n || !b || !faces || !x || !y || !z || !out || n[0] < 3 || n[1] < 3 || n[2] < 3) return LASTO_ERR_INVALID_ARG;
    const size_t N = (size_t)n[0] * n[1] * n[2];
    k_guess_features<<<blocks(N, 256), 256, 0, (cudaStream_t)stream>>>(n[0], n[1], n[2], b, faces, x, y, z, s0, s1,
                                                                       h_ref, out);
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

int lasto_nn_guess_grid(const int n[3], const float* pred, int ld, float scale, const double* faces, double* u,
                        void* stream)
{
    if (!n || !pred || !faces || !u || !(scale != 0.0f)) return LASTO_ERR_INVALID_ARG;
    const size_t N = (size_t)n[0] * n[1] * n[2];
    k_guess_grid<<<blocks(N, 256), 256, 0, (cudaStream_t)stream>>>(N, n[0], n[1], n[2], pred, ld, 1.0f / scale, faces,
                                                                   u);
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

int lasto_nn_adam(size_t n, float* w, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                  int step, void* w16, void* stream)
{
    if (step < 1) return LASTO_ERR_INVALID_ARG;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adam<<<blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(n, w, g, m, v, lr, b1, b2, eps, c1, c2, (bf16*)w16);
    return cudaGetLastError() == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

}  // extern "C"
