// Learned initial guess inside the solve graph.
//
// The paper starts every Poisson solve from nothing; here a small 3-D U-Net (trained on
// potentials this solver produced) predicts the potential on a 33^3 subgrid of the mesh
// (every m-th node per axis, m = (n - 1) / 32), and the prediction, carried up the multigrid
// hierarchy by the trilinear prolongation, is the first iterate.  Multigrid then runs to the
// same residual as from zero, so the network changes the iteration count only.
//
// Per cluster, after its right-hand side: restrict b (full weighting) down the hierarchy to
// the deepest level that still has at least 33 nodes per axis, resample it onto the 33^3
// subgrid (trilinear in physical coordinates; the identity when the level is the subgrid,
// as for 65^3, 129^3 and 257^3 meshes), take the subgrid's Dirichlet faces from the fine
// grid's (every subgrid and level node is a fine node), and write the network's input
// features.  Once every cluster's features are written, one batched forward pass runs.  Per
// cluster again: the predicted subgrid potential is resampled onto that level's interior,
// given its faces, and prolonged level by level to the fine grid, where it replaces the
// zero interior.
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace lasto {

namespace {

// (cin, cout, relu) of the 15 convolutions in order e1a e1b e2a e2b e3a e3b bta btb d3a d3b
// d2a d2b d1a d1b out: encoder 16-32-64-64 on 33, 17, 9, 5 nodes per axis, decoder on the
// concatenation [up-sampled coarser output, encoder output of the same level].
constexpr int NL = 15;
constexpr int L_CIN[NL] = {16, 16, 16, 32, 32, 64, 64, 64, 128, 64, 96, 32, 48, 16, 16};
constexpr int L_COUT[NL] = {16, 16, 32, 32, 64, 64, 64, 64, 64, 64, 32, 32, 16, 16, 16};
constexpr int L_RELU[NL] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 0};

__global__ void k_axis_stride(const double* __restrict__ src, int m, int n, double* __restrict__ dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[(size_t)i * m];
}

__device__ __forceinline__ int cell_below(const double* __restrict__ a, int n, double p)
{
    // largest i in [0, n-2] with a[i] <= p (clamped)
    int lo = 0, hi = n - 2;
    if (p <= a[0]) return 0;
    if (p >= a[n - 2]) return n - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// dst (grid B) = trilinear interpolation of src (grid A) in physical coordinates; both
// grids span the same box.  Exact (a copy) at the nodes B shares with A.  interior_only: B's
// faces are left as they are.
__global__ void k_resample(int ax_n, int ay_n, int az_n, const double* __restrict__ ax, const double* __restrict__ ay,
                           const double* __restrict__ az, const double* __restrict__ src, int bx_n, int by_n, int bz_n,
                           const double* __restrict__ bx, const double* __restrict__ by,
                           const double* __restrict__ bz, double* __restrict__ dst, int interior_only)
{
    const size_t N = (size_t)bx_n * by_n * bz_n;
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= N) return;
    const int i = (int)(t % bx_n), j = (int)((t / bx_n) % by_n), k = (int)(t / ((size_t)bx_n * by_n));
    if (interior_only && (i == 0 || j == 0 || k == 0 || i == bx_n - 1 || j == by_n - 1 || k == bz_n - 1)) return;
    const double px = bx[i], py = by[j], pz = bz[k];
    const int ci = cell_below(ax, ax_n, px), cj = cell_below(ay, ay_n, py), ck = cell_below(az, az_n, pz);
    const double tx = (px - ax[ci]) / (ax[ci + 1] - ax[ci]);
    const double ty = (py - ay[cj]) / (ay[cj + 1] - ay[cj]);
    const double tz = (pz - az[ck]) / (az[ck + 1] - az[ck]);
    const size_t sy = (size_t)ax_n, sz = (size_t)ax_n * ay_n;
    const double* c0 = src + (size_t)ck * sz + (size_t)cj * sy + ci;
    auto lerp = [](double a, double b, double w) { return w == 0.0 ? a : w == 1.0 ? b : a + w * (b - a); };
    const double v00 = lerp(c0[0], c0[1], tx), v01 = lerp(c0[sy], c0[sy + 1], tx);
    const double v10 = lerp(c0[sz], c0[sz + 1], tx), v11 = lerp(c0[sz + sy], c0[sz + sy + 1], tx);
    dst[t] = lerp(lerp(v00, v01, ty), lerp(v10, v11, ty), tz);
}

}  // namespace

// ---------------------------------------------------------------- network
struct GuessNet {
    int nbmax = 0;
    int dims[4] = {33, 17, 9, 5};
    size_t Ng[4] = {0, 0, 0, 0};   // nodes of one grid per level
    void* pool = nullptr;
    void* w16[NL] = {};
    float* bias[NL] = {};
    float scales[4] = {1, 1, 1, 1};   // s0, s1, h_ref, out
    // activations for nbmax grids
    float *x32, *e1, *cat1, *pred, *p1, *e2, *cat2, *d2, *p2, *e3, *cat3, *d3, *p3, *bt;
    float* scratch = nullptr;   // tap-group partial sums of the small-grid convolutions
    size_t scratch_floats = 0;
    void* wtmp = nullptr;       // BF16 weights of one layer before packing
    int* err = nullptr;         // tensor-core wait timeouts
    void *x16, *a0, *b0, *cat1h, *p1h, *a1, *cat2h, *p2h, *a2, *cat3h, *p3h, *a3;
};

size_t guess_param_count()
{
    size_t n = 0;
    for (int l = 0; l < NL; l++) n += (size_t)27 * L_CIN[l] * L_COUT[l] + L_COUT[l];
    return n;
}

void guess_net_free(GuessNet* g)
{
    if (!g) return;
    if (g->pool) cudaFree(g->pool);
    delete g;
}

int guess_net_create(const float* params, size_t n_params, const double scales[4], int nbmax, GuessNet** out,
                     cudaStream_t s)
{
    *out = nullptr;
    if (!params || !scales || n_params != guess_param_count() || nbmax < 1) return LASTO_ERR_INVALID_ARG;
    for (int q = 0; q < 4; q++)
        if (!(scales[q] == scales[q]) || scales[q] == 0.0) return LASTO_ERR_INVALID_ARG;
    GuessNet* g = new GuessNet();
    g->nbmax = nbmax;
    for (int l = 0; l < 4; l++) g->Ng[l] = (size_t)g->dims[l] * g->dims[l] * g->dims[l];
    for (int q = 0; q < 4; q++) g->scales[q] = (float)scales[q];
    // one pool: FP32 weights staging, BF16 weights, biases, activations
    const size_t nb = (size_t)nbmax, N0 = nb * g->Ng[0], N1 = nb * g->Ng[1], N2 = nb * g->Ng[2], N3 = nb * g->Ng[3];
    size_t f32 = n_params + 64, b16 = (size_t)27 * 128 * 64;
    for (int l = 0; l < NL; l++) b16 += (size_t)27 * L_CIN[l] * L_COUT[l];
    f32 += N0 * (16 + 16 + 48 + 16) + N1 * (16 + 32 + 96 + 32) + N2 * (32 + 64 + 128 + 64) + N3 * (64 + 64);
    b16 += N0 * (16 + 16 + 16 + 48) + N1 * (16 + 32 + 96) + N2 * (32 + 64 + 128) + N3 * (64 + 64);
    g->scratch_floats = (size_t)1216 * 64 * 128;
    f32 += g->scratch_floats;
    const size_t bytes = f32 * 4 + b16 * 2 + 64 * 256;
    if (cudaMalloc(&g->pool, bytes) != cudaSuccess) {
        delete g;
        return LASTO_ERR_NO_MEMORY;
    }
    unsigned char* p = static_cast<unsigned char*>(g->pool);
    auto take = [&](size_t nbytes) {
        void* r = p;
        p += (nbytes + 255) / 256 * 256;
        return r;
    };
    float* staging = (float*)take(n_params * 4);
    for (int l = 0; l < NL; l++) g->w16[l] = take((size_t)27 * L_CIN[l] * L_COUT[l] * 2);
    for (int l = 0; l < NL; l++) g->bias[l] = (float*)take((size_t)L_COUT[l] * 4);
    auto F = [&](size_t n) { return (float*)take(n * 4); };
    auto H = [&](size_t n) { return take(n * 2); };
    g->x32 = F(N0 * 16); g->e1 = F(N0 * 16); g->cat1 = F(N0 * 48); g->pred = F(N0 * 16);
    g->p1 = F(N1 * 16); g->e2 = F(N1 * 32); g->cat2 = F(N1 * 96); g->d2 = F(N1 * 32);
    g->p2 = F(N2 * 32); g->e3 = F(N2 * 64); g->cat3 = F(N2 * 128); g->d3 = F(N2 * 64);
    g->p3 = F(N3 * 64); g->bt = F(N3 * 64);
    g->x16 = H(N0 * 16); g->a0 = H(N0 * 16); g->b0 = H(N0 * 16); g->cat1h = H(N0 * 48);
    g->p1h = H(N1 * 16); g->a1 = H(N1 * 32); g->cat2h = H(N1 * 96);
    g->p2h = H(N2 * 32); g->a2 = H(N2 * 64); g->cat3h = H(N2 * 128);
    g->p3h = H(N3 * 64); g->a3 = H(N3 * 64);
    g->scratch = F(g->scratch_floats);
    g->wtmp = H((size_t)27 * 128 * 64);
    g->err = (int*)take(256);
    cudaError_t e = cudaMemcpyAsync(staging, params, n_params * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->err, 0, sizeof(int), s);
    size_t off = 0;
    for (int l = 0; l < NL && e == cudaSuccess; l++) {
        const size_t nw = (size_t)27 * L_CIN[l] * L_COUT[l];
        // BF16 weights of the layer, packed into the per-step operand tiles the tensor-core
        // convolution reads
        if (lasto_nn_to_bf16(nw, staging + off, g->wtmp, s) != LASTO_OK) e = cudaErrorLaunchFailure;
        if (e == cudaSuccess) e = launch_pack_weights(L_CIN[l], L_COUT[l], g->wtmp, g->w16[l], s);
        off += nw;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->bias[l], staging + off, (size_t)L_COUT[l] * 4, cudaMemcpyDeviceToDevice, s);
        off += L_COUT[l];
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        guess_net_free(g);
        return LASTO_ERR_CUDA;
    }
    *out = g;
    return LASTO_OK;
}

float* guess_net_features(GuessNet* g, int k) { return g->x32 + (size_t)k * g->Ng[0] * 16; }
const float* guess_net_prediction(GuessNet* g, int k) { return g->pred + (size_t)k * g->Ng[0] * 16; }
int guess_net_capacity(const GuessNet* g) { return g ? g->nbmax : 0; }
const float* guess_net_scales(const GuessNet* g) { return g->scales; }

// Forward pass over grids 0 .. nb-1 of the feature buffer on the tcgen05 convolution; the
// prediction is channel 0 of pred ([node][16]).
int guess_net_forward(GuessNet* g, int nb, cudaStream_t s)
{
    if (nb < 1 || nb > g->nbmax) return LASTO_ERR_INVALID_ARG;
    const size_t N0 = nb * g->Ng[0], N1 = nb * g->Ng[1], N2 = nb * g->Ng[2], N3 = nb * g->Ng[3];
    int dim[4][3];
    for (int l = 0; l < 4; l++) dim[l][0] = dim[l][1] = dim[l][2] = g->dims[l];
    int st = LASTO_OK;
    auto conv = [&](int l, int lv, const void* x, float* y32, int ldy32, int off32, void* y16, int ldy16, int off16) {
        if (st) return;
        st = conv_fwd_tc(nb, dim[lv], L_CIN[l], L_COUT[l], x, g->w16[l], g->bias[l], L_RELU[l], y32, ldy32, off32, y16,
                         ldy16, off16, g->scratch, g->scratch_floats, g->err, s);
    };
    auto tobf = [&](size_t n, const float* a, void* b) {
        if (!st) st = lasto_nn_to_bf16(n, a, b, s);
    };
    auto down = [&](int lv, int C, const float* x, float* y) {
        if (!st) st = lasto_nn_down(nb, dim[lv], C, x, y, 0, s);
    };
    auto up = [&](int lv_fine, int C, const float* x, float* y, int ldy) {
        if (!st) st = lasto_nn_up(nb, dim[lv_fine], C, x, y, ldy, 0, 0, s);
    };
    auto copy = [&](size_t nodes, int C, const float* src, float* dst, int ldd, int doff) {
        if (!st) st = lasto_nn_copy_channels(nodes, C, src, C, 0, dst, ldd, doff, 0, s);
    };
    tobf(N0 * 16, g->x32, g->x16);
    conv(0, 0, g->x16, nullptr, 0, 0, g->a0, 16, 0);          // e1a
    conv(1, 0, g->a0, g->e1, 16, 0, nullptr, 0, 0);           // e1b
    down(0, 16, g->e1, g->p1);
    tobf(N1 * 16, g->p1, g->p1h);
    conv(2, 1, g->p1h, nullptr, 0, 0, g->a1, 32, 0);          // e2a
    conv(3, 1, g->a1, g->e2, 32, 0, nullptr, 0, 0);           // e2b
    down(1, 32, g->e2, g->p2);
    tobf(N2 * 32, g->p2, g->p2h);
    conv(4, 2, g->p2h, nullptr, 0, 0, g->a2, 64, 0);          // e3a
    conv(5, 2, g->a2, g->e3, 64, 0, nullptr, 0, 0);           // e3b
    down(2, 64, g->e3, g->p3);
    tobf(N3 * 64, g->p3, g->p3h);
    conv(6, 3, g->p3h, nullptr, 0, 0, g->a3, 64, 0);          // bta
    conv(7, 3, g->a3, g->bt, 64, 0, nullptr, 0, 0);           // btb
    up(2, 64, g->bt, g->cat3, 128);                           // [up(bt), e3]
    copy(N2, 64, g->e3, g->cat3, 128, 64);
    tobf(N2 * 128, g->cat3, g->cat3h);
    conv(8, 2, g->cat3h, nullptr, 0, 0, g->a2, 64, 0);        // d3a
    conv(9, 2, g->a2, g->d3, 64, 0, nullptr, 0, 0);           // d3b
    up(1, 64, g->d3, g->cat2, 96);                            // [up(d3), e2]
    copy(N1, 32, g->e2, g->cat2, 96, 64);
    tobf(N1 * 96, g->cat2, g->cat2h);
    conv(10, 1, g->cat2h, nullptr, 0, 0, g->a1, 32, 0);       // d2a
    conv(11, 1, g->a1, g->d2, 32, 0, nullptr, 0, 0);          // d2b
    up(0, 32, g->d2, g->cat1, 48);                            // [up(d2), e1]
    copy(N0, 16, g->e1, g->cat1, 48, 32);
    tobf(N0 * 48, g->cat1, g->cat1h);
    conv(12, 0, g->cat1h, nullptr, 0, 0, g->a0, 16, 0);       // d1a
    conv(13, 0, g->a0, nullptr, 0, 0, g->b0, 16, 0);          // d1b
    conv(14, 0, g->b0, g->pred, 16, 0, nullptr, 0, 0);        // out (no ReLU)
    return st;
}

cudaError_t launch_axis_stride(const double* src, int m, int n, double* dst, cudaStream_t s)
{
    k_axis_stride<<<(n + 127) / 128, 128, 0, s>>>(src, m, n, dst);
    return cudaGetLastError();
}

cudaError_t launch_resample(const int na[3], const double* ax, const double* ay, const double* az, const double* src,
                            const int nbn[3], const double* bx, const double* by, const double* bz, double* dst,
                            int interior_only, cudaStream_t s)
{
    const size_t N = (size_t)nbn[0] * nbn[1] * nbn[2];
    k_resample<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(na[0], na[1], na[2], ax, ay, az, src, nbn[0], nbn[1], nbn[2],
                                                           bx, by, bz, dst, interior_only);
    return cudaGetLastError();
}

}  // namespace lasto
