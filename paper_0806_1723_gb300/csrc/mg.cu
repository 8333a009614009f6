// Multigrid and conjugate-gradient kernels of the interstitial Poisson solve
// (Section 3: "a finite difference scheme and a multigrid method").
//
// All kernels walk the grid with a flat node index.  Every smoothed level has an
// odd number of nodes per axis, so the parity of the flat index equals the parity
// of i+j+k: red nodes are the even flat indices, and a half sweep is one thread per
// node of that colour with unit-stride neighbour loads.  Reductions are two-stage
// (per-block partials, then one block in a fixed order), so every norm and dot is
// bitwise reproducible.
#include <algorithm>

#include "internal.cuh"
#include "ctl.cuh"
#include "stage.cuh"

namespace lasto {

constexpr int NT = 256;

// Flat index -> (i, j, k).  Grids hold fewer than 2^31 nodes (checked where they are accepted),
// so the decomposition divides by the level's invariant nx and nx * ny with a multiply-high and
// a shift (LevelT's division constants): a hardware-less integer division would cost more than
// the stencil update it indexes.
template <typename T>
__device__ __forceinline__ void node_ijk(size_t P, const LevelT<T>& L, int& i, int& j, int& k)
{
    const unsigned p = (unsigned)P;
    const unsigned kk = div_by(p, L.dvxy), rem = p - kk * ((unsigned)L.nx * (unsigned)L.ny);
    const unsigned jj = div_by(rem, L.dvx);
    k = (int)kk;
    j = (int)jj;
    i = (int)(rem - jj * (unsigned)L.nx);
}

template <typename T>
__device__ __forceinline__ bool is_face(const LevelT<T>& L, int i, int j, int k)
{
    return i == 0 || j == 0 || k == 0 || i == L.nx - 1 || j == L.ny - 1 || k == L.nz - 1;
}

// sum of the six neighbour terms in the fixed order x-, x+, y-, y+, z-, z+
// (neighbours addressed from the node's own pointer with 32-bit offsets: a plane holds fewer
// than 2^31 nodes)
// LS = 1: colour-split storage (LevelT): the neighbours all sit in the other colour's half, at
// (P +- d) >> 1.  The terms and their order are the same in both storage orders.
template <int LS = 0, typename T>
__device__ __forceinline__ T offdiag(const LevelT<T>& L, const T* __restrict__ u, size_t P, int i, int j, int k)
{
    if constexpr (LS == 0) {
        const int sy = L.nx, sz = L.nx * L.ny;
        const T* __restrict__ c = u + P;
        T t = L.ax[0].cm[i] * c[-1];
        t = fma(L.ax[0].cp[i], c[1], t);
        t = fma(L.ax[1].cm[j], c[-sy], t);
        t = fma(L.ax[1].cp[j], c[sy], t);
        t = fma(L.ax[2].cm[k], c[-sz], t);
        t = fma(L.ax[2].cp[k], c[sz], t);
        return t;
    } else {
        const unsigned p = (unsigned)P, sy = (unsigned)L.nx, sz = (unsigned)L.nx * (unsigned)L.ny;
        const T* __restrict__ o = u + (size_t)(1u - (p & 1u)) * L.H;
        T t = L.ax[0].cm[i] * o[(p - 1u) >> 1];
        t = fma(L.ax[0].cp[i], o[(p + 1u) >> 1], t);
        t = fma(L.ax[1].cm[j], o[(p - sy) >> 1], t);
        t = fma(L.ax[1].cp[j], o[(p + sy) >> 1], t);
        t = fma(L.ax[2].cm[k], o[(p - sz) >> 1], t);
        t = fma(L.ax[2].cp[k], o[(p + sz) >> 1], t);
        return t;
    }
}

// storage position of node P for a compile-time storage order
template <int LS, typename T>
__device__ __forceinline__ unsigned pos(const LevelT<T>& L, size_t P)
{
    if constexpr (LS == 0) return (unsigned)P;
    else return ((unsigned)P >> 1) + ((unsigned)P & 1u) * L.H;
}

template <typename T>
__device__ __forceinline__ T dsum(const LevelT<T>& L, int i, int j, int k)
{
    return L.ax[0].dg[i] + L.ax[1].dg[j] + L.ax[2].dg[k];
}

// ---------------------------------------------------------------- smoother
// (LS = 1: colour-split storage, FP32 only; thread t's node is then at t + colour H, so every
// load and store of a warp is one unit-stride run)
template <typename T, int LS>
__device__ __forceinline__ void k_rbgs_body(LevelT<T> L, T* __restrict__ u, const T* __restrict__ b, int colour, size_t nhalf)
{
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;   // nodes < 2^31
    if (t >= (unsigned)nhalf) return;
    const unsigned P = 2 * t + colour;
    int i, j, k;
    node_ijk(P, L, i, j, k);
    if (is_face(L, i, j, k)) return;
    const unsigned Q = pos<LS>(L, P);
    const T acc = b[Q] - offdiag<LS>(L, u, P, i, j, k);
    if constexpr (sizeof(T) == 8) {
        u[Q] = acc * L.inv_diag[P];
    } else {
        u[Q] = rb_point32(acc, dsum(L, i, j, k));
    }
}

// The first (red) FP32 half sweep from u = 0: every neighbour term is +0, so the update is the
// point value rb_point32(b, diagonal) -- bitwise the half sweep's result -- and reads neither u
// nor the black nodes, which the black half sweep after it overwrites without reading.  VU red
// nodes per thread, loads first.  (The faces of u must already be zero.)
template <int LS>
__global__ void __launch_bounds__(256) k_first_red32(LevelT<float> L, float* __restrict__ u, const float* __restrict__ b,
                                                     unsigned nred)
{
    constexpr int NV = 4;
    const unsigned t0 = blockIdx.x * (256u * NV) + threadIdx.x;
    float bv[NV];
    unsigned Q[NV];
    bool on[NV];
#pragma unroll
    for (int q = 0; q < NV; q++) {
        const unsigned t = t0 + 256u * q;
        on[q] = false;
        bv[q] = 0.0f;
        Q[q] = 0u;
        if (t < nred) {
            int i, j, k;
            node_ijk(2 * (size_t)t, L, i, j, k);
            if (!is_face(L, i, j, k)) {
                on[q] = true;
                Q[q] = LS ? t : 2u * t;
                bv[q] = b[Q[q]];
                bv[q] = rb_point32(bv[q], dsum(L, i, j, k));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NV; q++)
        if (on[q]) u[Q[q]] = bv[q];
}

cudaError_t launch_first_red32(const LevelT<float>& L, float* u, const float* b, cudaStream_t s)
{
    const unsigned nred = (unsigned)((L.N() + 1) / 2);
    const unsigned g = (nred + 256u * 4u - 1u) / (256u * 4u);
    if (L.lsh)
        k_first_red32<1><<<g, 256, 0, s>>>(L, u, b, nred);
    else
        k_first_red32<0><<<g, 256, 0, s>>>(L, u, b, nred);
    return cudaGetLastError();
}

template <typename T, int LS>
__global__ void __launch_bounds__(512) k_rbgs(LevelT<T> L, T* __restrict__ u, const T* __restrict__ b, int colour, size_t nhalf)
{
    k_rbgs_body<T, LS>(L, u, b, colour, nhalf);
}

// The same half sweep with one block per interior (j, k) row and one thread per node of the
// colour along i: no index division, the row's y and z coefficients the same in every thread.
// The node update is k_rbgs's expression, so the two are bitwise equal.
template <typename T, int LS>
__global__ void __launch_bounds__(512) k_rbgs_row(LevelT<T> L, T* __restrict__ u, const T* __restrict__ b, int colour)
{
    const int j = blockIdx.x + 1, k = blockIdx.y + 1;
    const int i = 2 * (int)threadIdx.x + ((colour + j + k) & 1);   // flat-index parity = parity of i + j + k
    if (i == 0 || i >= L.nx - 1) return;
    const unsigned P = ((unsigned)k * L.ny + j) * L.nx + i;   // nodes < 2^31
    const unsigned Q = pos<LS>(L, P);
    const T acc = b[Q] - offdiag<LS>(L, u, P, i, j, k);
    if constexpr (sizeof(T) == 8) {
        u[Q] = acc * L.inv_diag[P];
    } else {
        u[Q] = rb_point32(acc, dsum(L, i, j, k));
    }
}

// The FP32 half sweep over colour-split storage with one warp per interior (j, k) row: lane l
// updates the row's interior nodes of the colour numbered l, l + 32, ..., l + 32 (V - 1) in x
// order, so every load and store of the warp is one unit-stride run.  The row's y and z
// coefficients, its flat index and the six neighbour offsets (row constants in this storage:
// node q of the colour has its neighbours at q + d in the other colour's half) are formed once
// per row.  A row's own right-hand side and the other colour's row one plane further on (where
// the sweep first touches it, as a z+ neighbour; its other reads then hit L2) are prefetched
// into L2 `pf` rows ahead, about half a wave of resident warps, which keeps more DRAM requests
// in flight than the warps' own loads do.  The node update is k_rbgs's expression, so the two
// are bitwise equal.
template <int V>
__device__ __forceinline__ void k_rbgs_split_rows_body(LevelT<float> L, float* __restrict__ u, const float* __restrict__ b, int colour, int pf)
{
    const int my = L.ny - 2;
    const int row = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    if (row >= my * (L.nz - 2)) return;
    const int lane = threadIdx.x & 31;
    const int k = row / my + 1, j = row - (k - 1) * my + 1;
    const int nx = L.nx;
    const unsigned nxy = (unsigned)nx * (unsigned)L.ny;
    const int c = colour;
    const int i1 = ((c + j + k) & 1) ? 1 : 2;             // first interior node of the colour
    const int cnt = (nx - i1) >> 1;                        // interior nodes of the colour in the row
    const unsigned q0 = ((unsigned)k * nxy + (unsigned)j * (unsigned)nx + (unsigned)i1) >> 1;
    const int hx = (nx - 1) >> 1, hxy = (int)((nxy - 1) >> 1);
    const int dxm = c - 1, dxp = c, dym = c - 1 - hx, dyp = c + hx, dzm = c - 1 - hxy, dzp = c + hxy;
    // lane l's nodes are l + 32 v from q0: one base pointer per operand stream, so every load and
    // store below is that base plus a compile-time offset (no per-node address arithmetic)
    const float* __restrict__ o = u + (size_t)(1 - c) * L.H + q0 + lane;   // the other colour
    const float* __restrict__ nxm = o + dxm;
    const float* __restrict__ nxp = o + dxp;
    const float* __restrict__ nym = o + dym;
    const float* __restrict__ nyp = o + dyp;
    const float* __restrict__ nzm = o + dzm;
    const float* __restrict__ nzp = o + dzp;
    float* __restrict__ uo = u + (size_t)c * L.H + q0 + lane;
    const float* __restrict__ bo = b + (size_t)c * L.H + q0 + lane;
    const float cmy = L.ax[1].cm[j], cpy = L.ax[1].cp[j], dgy = L.ax[1].dg[j];
    const float cmz = L.ax[2].cm[k], cpz = L.ax[2].cp[k], dgz = L.ax[2].dg[k];
    const float* __restrict__ cmx = L.ax[0].cm + i1 + 2 * lane;
    const float* __restrict__ cpx = L.ax[0].cp + i1 + 2 * lane;
    const float* __restrict__ dgx = L.ax[0].dg + i1 + 2 * lane;
    if (row + pf < my * (L.nz - 2)) {
        // (an interior row's lines, up to 31 values past its end: still inside the array, as
        // the face plane follows)
        const int r2 = row + pf;
        const int k2 = r2 / my + 1, j2 = r2 - (k2 - 1) * my + 1;
        const int i2 = ((c + j2 + k2) & 1) ? 1 : 2;
        const unsigned q2 = ((unsigned)k2 * nxy + (unsigned)j2 * (unsigned)nx + (unsigned)i2) >> 1;
        if (lane <= (cnt + 31) / 32) {
            const float* pb = b + (size_t)c * L.H + q2 + 32 * lane;
            const float* pz = u + (size_t)(1 - c) * L.H + q2 + dzp + 32 * lane;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(pb));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(pz));
        }
    }
    const int left = cnt - lane;
#pragma unroll
    for (int v = 0; v < V; v++) {
        if (32 * v < left) {
            float t = cmx[64 * v] * nxm[32 * v];
            t = fmaf(cpx[64 * v], nxp[32 * v], t);
            t = fmaf(cmy, nym[32 * v], t);
            t = fmaf(cpy, nyp[32 * v], t);
            t = fmaf(cmz, nzm[32 * v], t);
            t = fmaf(cpz, nzp[32 * v], t);
            const float acc = bo[32 * v] - t;
            uo[32 * v] = rb_point32(acc, dgx[64 * v] + dgy + dgz);
        }
    }
}

template <int V>
__global__ void __launch_bounds__(256) k_rbgs_split_rows(LevelT<float> L, float* __restrict__ u, const float* __restrict__ b, int colour, int pf)
{
    k_rbgs_split_rows_body<V>(L, u, b, colour, pf);
}

// prefetch distance of the row-per-warp sweep: half the rows the device holds resident
// (cached per device)
template <int V>
cudaError_t split_rows_pf(int* pf)
{
    static int pf_rows[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (pf_rows[dev] == 0) {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rbgs_split_rows<V>, 256, 0);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        pf_rows[dev] = std::max(1, per_sm * sms * 8 / 2);
    }
    *pf = pf_rows[dev];
    return cudaSuccess;
}

template <int V>
cudaError_t launch_split_rows_v(const LevelT<float>& L, float* u, const float* b, int colour, cudaStream_t s)
{
    int pf = 0;
    const cudaError_t e = split_rows_pf<V>(&pf);
    if (e != cudaSuccess) return e;
    const int rows = (L.ny - 2) * (L.nz - 2);
    k_rbgs_split_rows<V><<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(L, u, b, colour, pf);
    return cudaGetLastError();
}

// nodes of one colour per interior row, in units of 32 (0: too long for the row-per-warp kernel)
inline int split_rows_v(int nx) { return (nx - 1) / 2 <= 256 ? std::max(1, ((nx - 1) / 2 + 31) / 32) : 0; }

// nt > 0: k_rbgs with nt threads per block; nt == 0: k_rbgs_row (rows of at most 1023 nodes),
// over colour-split storage k_rbgs_split_rows (rows of at most 513 nodes)
template <typename T>
cudaError_t launch_rbgs(const LevelT<T>& L, T* u, const T* b, int colour, cudaStream_t s, int nt, int* status)
{
    const bool split = L.lsh != 0;
    if (split && sizeof(T) != 4) return cudaErrorInvalidValue;   // FP64 levels keep natural storage
    if (nt == RBGS_STAGED) {
        if constexpr (sizeof(T) == 4) {
            if (split) return launch_split_stage(L, u, b, colour, status, s);
        }
        return cudaErrorInvalidValue;
    }
    if (nt == 0 && split) {
        if constexpr (sizeof(T) == 4) {
            if (L.ny < 3 || L.nz < 3) return cudaErrorInvalidValue;
            switch (split_rows_v(L.nx)) {
                case 1: return launch_split_rows_v<1>(L, u, b, colour, s);
                case 2: return launch_split_rows_v<2>(L, u, b, colour, s);
                case 3: return launch_split_rows_v<3>(L, u, b, colour, s);
                case 4: return launch_split_rows_v<4>(L, u, b, colour, s);
                case 5: return launch_split_rows_v<5>(L, u, b, colour, s);
                case 6: return launch_split_rows_v<6>(L, u, b, colour, s);
                case 7: return launch_split_rows_v<7>(L, u, b, colour, s);
                case 8: return launch_split_rows_v<8>(L, u, b, colour, s);
                default: return cudaErrorInvalidValue;
            }
        }
    }
    if (nt == 0) {
        const int th = ((L.nx + 1) / 2 + 31) / 32 * 32;
        if (th > 512 || L.ny < 3 || L.nz < 3 || L.nz - 2 > 65535) return cudaErrorInvalidValue;
        const dim3 g((unsigned)(L.ny - 2), (unsigned)(L.nz - 2));
        if (split)
            k_rbgs_row<T, 1><<<g, th, 0, s>>>(L, u, b, colour);
        else
            k_rbgs_row<T, 0><<<g, th, 0, s>>>(L, u, b, colour);
        return cudaGetLastError();
    }
    if (nt < 32 || nt > 512 || nt % 32) return cudaErrorInvalidValue;
    const size_t N = L.N();
    const size_t nhalf = (N + 1 - colour) / 2;
    const unsigned g = (unsigned)((nhalf + nt - 1) / nt);
    if (split)
        k_rbgs<T, 1><<<g, nt, 0, s>>>(L, u, b, colour, nhalf);
    else
        k_rbgs<T, 0><<<g, nt, 0, s>>>(L, u, b, colour, nhalf);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- residual / apply
template <typename T>
__global__ void __launch_bounds__(NT) k_residual(LevelT<T> L, const T* __restrict__ u, const T* __restrict__ b,
                                                T* __restrict__ r)
{
    const size_t P = blockIdx.x * (size_t)NT + threadIdx.x;
    if (P >= L.N()) return;
    int i, j, k;
    node_ijk(P, L, i, j, k);
    if (is_face(L, i, j, k)) {
        r[P] = T(0);
        return;
    }
    const T Au = fma(-dsum(L, i, j, k), u[P], offdiag(L, u, P, i, j, k));
    r[P] = b[P] - Au;
}

template <typename T>
__global__ void __launch_bounds__(NT) k_apply(LevelT<T> L, const T* __restrict__ u, T* __restrict__ Au)
{
    const size_t P = blockIdx.x * (size_t)NT + threadIdx.x;
    if (P >= L.N()) return;
    int i, j, k;
    node_ijk(P, L, i, j, k);
    Au[P] = is_face(L, i, j, k) ? T(0) : fma(-dsum(L, i, j, k), u[P], offdiag(L, u, P, i, j, k));
}

template <typename T>
cudaError_t launch_residual(const LevelT<T>& L, const T* u, const T* b, T* r, cudaStream_t s)
{
    if (L.lsh) return cudaErrorInvalidValue;   // natural storage only
    k_residual<T><<<(unsigned)((L.N() + NT - 1) / NT), NT, 0, s>>>(L, u, b, r);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(const LevelT<T>& L, const T* u, T* Au, cudaStream_t s)
{
    if (L.lsh) return cudaErrorInvalidValue;
    k_apply<T><<<(unsigned)((L.N() + NT - 1) / NT), NT, 0, s>>>(L, u, Au);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- transfers
// bc = Vc^-1 P^T Vf r: the 27-point stencil factorises into per-axis weights.
template <typename T>
__global__ void __launch_bounds__(NT) k_restrict(LevelT<T> F, LevelT<T> C, const T* __restrict__ r,
                                                T* __restrict__ bc)
{
    const size_t t = blockIdx.x * (size_t)NT + threadIdx.x;
    if (t >= C.N()) return;
    int I, J, K;
    node_ijk(t, C, I, J, K);
    if (is_face(C, I, J, K)) {
        bc[t] = T(0);
        return;
    }
    const T* wx = F.ax[0].rw + 3 * I;
    const T* wy = F.ax[1].rw + 3 * J;
    const T* wz = F.ax[2].rw + 3 * K;
    const size_t sy = F.nx, sz = (size_t)F.nx * F.ny;
    const T* base = r + (size_t)(2 * K - 1) * sz + (size_t)(2 * J - 1) * sy + (2 * I - 1);
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int bb = 0; bb < 3; bb++) {
            const T* row = base + c * sz + bb * sy;
            const T s = fma(wx[0], row[0], fma(wx[1], row[1], wx[2] * row[2]));
            acc = fma(wz[c] * wy[bb], s, acc);
        }
    bc[t] = acc;
}

template <typename T>
cudaError_t launch_restrict(const LevelT<T>& F, const LevelT<T>& C, const T* r, T* bc, cudaStream_t s)
{
    if (F.lsh || C.lsh) return cudaErrorInvalidValue;
    k_restrict<T><<<(unsigned)((C.N() + NT - 1) / NT), NT, 0, s>>>(F, C, r, bc);
    return cudaGetLastError();
}

// u += P ec: per axis an even fine node sits on a coarse node (weight 1), an odd one
// between two (weights pl, pr in physical coordinates).
template <typename T, int LS>
__global__ void __launch_bounds__(NT) k_prolong_add(LevelT<T> F, LevelT<T> C, const T* __restrict__ ec,
                                                   T* __restrict__ u)
{
    const size_t P = blockIdx.x * (size_t)NT + threadIdx.x;
    if (P >= F.N()) return;
    int i, j, k;
    node_ijk(P, F, i, j, k);
    if (is_face(F, i, j, k)) return;
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nk = (k & 1) ? 2 : 1;
    const T wx[2] = {F.ax[0].pl[i], F.ax[0].pr[i]};
    const T wy[2] = {F.ax[1].pl[j], F.ax[1].pr[j]};
    const T wz[2] = {F.ax[2].pl[k], F.ax[2].pr[k]};
    const size_t sy = C.nx, sz = (size_t)C.nx * C.ny;
    const T* base = ec + (size_t)K * sz + (size_t)J * sy + I;
    T e = T(0);
    for (int c = 0; c < nk; c++)
        for (int bb = 0; bb < nj; bb++) {
            const T* row = base + c * sz + bb * sy;
            const T s = (ni == 2) ? fma(wx[0], row[0], wx[1] * row[1]) : row[0];
            e = fma(wz[c] * wy[bb], s, e);
        }
    u[pos<LS>(F, P)] += e;
}

// The same in FP32 with one warp per interior fine (j, k) row, lanes along the row's red nodes and
// its black ones: the row's y and z weights and coarse rows once per warp, no index division; the
// node expression is k_prolong_add's, so the two are bitwise equal.  A lane takes PU nodes of each
// colour run (64 fine nodes apart) per step and loads all their fine values before the first
// update, so 2 PU loads of the iterate are in flight per lane rather than one.
constexpr int PU = 3;

// L2 bulk prefetch of the fine row `row` of a row-per-warp kernel (both colours), by one lane:
// the run is widened to whole 16-byte units inside the array
template <int LS>
__device__ __forceinline__ void prefetch_row(const LevelT<float>& F, const float* a, int row)
{
    const int my = F.ny - 2;
    const int k = row / my + 1, j = row - (k - 1) * my + 1;
    const unsigned P = ((unsigned)k * (unsigned)F.ny + (unsigned)j) * (unsigned)F.nx, N = (unsigned)F.N();
    for (int t = 0; t < (LS ? 2 : 1); t++) {
        const unsigned lo = LS ? (unsigned)t * F.H + (P >> 1) : P;
        const unsigned hi = LS ? (unsigned)t * F.H + ((P + (unsigned)F.nx) >> 1) + 1u : P + (unsigned)F.nx;
        const unsigned a0 = lo & ~3u, a1 = min((hi + 3u) & ~3u, N & ~3u);
        if (a1 > a0) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(a + a0), "r"((a1 - a0) * 4u) : "memory");
    }
}

template <int LS>
__device__ __forceinline__ void k_prolong_add_rows_body(LevelT<float> F, LevelT<float> C, const float* __restrict__ ec, float* __restrict__ u, int pf)
{
    const int my = F.ny - 2;
    const int row = (int)(blockIdx.x * 8 + (threadIdx.x >> 5));
    if (row >= my * (F.nz - 2)) return;
    const int lane = threadIdx.x & 31;
    if (pf > 0 && lane == 0 && row + pf < my * (F.nz - 2)) prefetch_row<LS>(F, u, row + pf);
    const int k = row / my + 1, j = row - (k - 1) * my + 1;
    const int nj = (j & 1) ? 2 : 1, nk = (k & 1) ? 2 : 1;
    const float wy[2] = {F.ax[1].pl[j], F.ax[1].pr[j]};
    const float wz[2] = {F.ax[2].pl[k], F.ax[2].pr[k]};
    const size_t sy = C.nx, sz = (size_t)C.nx * C.ny;
    const float* __restrict__ crow = ec + (size_t)(k >> 1) * sz + (size_t)(j >> 1) * sy;
    const unsigned f0 = ((unsigned)k * (unsigned)F.ny + (unsigned)j) * (unsigned)F.nx;
    // the red nodes of the row, then the black ones (unit stride over colour-split storage); the
    // parity of i, and with it the x stencil, is the same along a run
    for (int m0 = 0; 64 * m0 < F.nx; m0 += PU) {
        float uv[2][PU];
        unsigned Q[2][PU];
        bool ok[2][PU];
#pragma unroll
        for (int t = 0; t < 2; t++)
#pragma unroll
            for (int m = 0; m < PU; m++) {
                const int i = (((t + j + k) & 1) ? 1 : 2) + 2 * lane + 64 * (m0 + m);
                ok[t][m] = i < F.nx - 1;
                Q[t][m] = pos<LS>(F, f0 + (unsigned)i);
                uv[t][m] = ok[t][m] ? u[Q[t][m]] : 0.0f;
            }
#pragma unroll
        for (int t = 0; t < 2; t++)
#pragma unroll
            for (int m = 0; m < PU; m++) {
                if (!ok[t][m]) continue;
                const int i = (((t + j + k) & 1) ? 1 : 2) + 2 * lane + 64 * (m0 + m);
                const int ni = (i & 1) ? 2 : 1;
                const float wx[2] = {F.ax[0].pl[i], F.ax[0].pr[i]};
                const float* base = crow + (i >> 1);
                float e = 0.0f;
#pragma unroll
                for (int c = 0; c < 2; c++)
#pragma unroll
                    for (int bb = 0; bb < 2; bb++) {
                        if (c >= nk || bb >= nj) continue;
                        const float* r = base + c * sz + bb * sy;
                        const float sv = (ni == 2) ? fmaf(wx[0], r[0], wx[1] * r[1]) : r[0];
                        e = fmaf(wz[c] * wy[bb], sv, e);
                    }
                u[Q[t][m]] = uv[t][m] + e;
            }
    }
}

template <int LS>
__global__ void __launch_bounds__(256) k_prolong_add_rows(LevelT<float> F, LevelT<float> C, const float* __restrict__ ec, float* __restrict__ u, int pf)
{
    k_prolong_add_rows_body<LS>(F, C, ec, u, pf);
}

// prefetch distance of the row-per-warp prolongation: half the rows the device holds resident
// (none on small levels, whose rows stay in L2 anyway)
template <int LS>
static cudaError_t prolong_rows_pf(const LevelT<float>& F, int* pf)
{
    static int pf_rows[64] = {0};
    *pf = 0;
    if (F.N() < (size_t(1) << 22)) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (pf_rows[dev] == 0) {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prolong_add_rows<LS>, 256, 0);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        pf_rows[dev] = std::max(1, per_sm * sms * 8 / 2);
    }
    *pf = pf_rows[dev];
    return cudaSuccess;
}

// (the fine level in either storage order, the coarse one natural)
template <typename T>
cudaError_t launch_prolong_add(const LevelT<T>& F, const LevelT<T>& C, const T* ec, T* u, cudaStream_t s, int* status)
{
    if (C.lsh) return cudaErrorInvalidValue;
    if constexpr (sizeof(T) == 4) {
        // colour-split fine level: the plane-staged form (bitwise the same); the solver's arrays
        // are padded to 256 bytes, so ec is readable to the next 16 bytes past its end
        if (F.lsh && split_stage_ok(F.nx, F.ny, F.nz) && !((uintptr_t)u & 15u) && !((uintptr_t)ec & 15u))
            return launch_prolong_stage(F, C, ec, u, status, s);
        if (F.ny >= 3 && F.nz >= 3) {
            const unsigned g = (unsigned)(((size_t)(F.ny - 2) * (F.nz - 2) + 7) / 8);
            int pf = 0;
            const cudaError_t e = F.lsh ? prolong_rows_pf<1>(F, &pf) : prolong_rows_pf<0>(F, &pf);
            if (e != cudaSuccess) return e;
            if ((uintptr_t)u & 15u) pf = 0;
            if (F.lsh)
                k_prolong_add_rows<1><<<g, 256, 0, s>>>(F, C, ec, u, pf);
            else
                k_prolong_add_rows<0><<<g, 256, 0, s>>>(F, C, ec, u, pf);
            return cudaGetLastError();
        }
    }
    const unsigned g = (unsigned)((F.N() + NT - 1) / NT);
    if (F.lsh)
        k_prolong_add<T, 1><<<g, NT, 0, s>>>(F, C, ec, u);
    else
        k_prolong_add<T, 0><<<g, NT, 0, s>>>(F, C, ec, u);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- exact coarse solve
constexpr int MC = MAX_COARSE - 2;
constexpr int MC3 = MC * MC * MC;

// Exact solve on the coarsest grid by fast diagonalisation; one thread block, s0/s1 are
// shared buffers of MC3 doubles.  add = 1: e += A^-1 b; add = 0: e = A^-1 b with zero faces.
template <typename T>
__device__ void coarse_apply_block(const LevelT<T>& L, const CoarseEig* __restrict__ E, const T* __restrict__ b,
                                   T* __restrict__ e, int add, double* s0, double* s1)
{
    const int mx = L.nx - 2, my = L.ny - 2, mz = L.nz - 2, M = mx * my * mz;
    const size_t sy = L.nx, sz = (size_t)L.nx * L.ny;
    auto node = [&](int a, int bb, int c) { return (size_t)(c + 1) * sz + (size_t)(bb + 1) * sy + (a + 1); };
    for (int t = threadIdx.x; t < M; t += blockDim.x) {
        const int a = t % mx, bb = (t / mx) % my, c = t / (mx * my);
        s0[t] = (double)b[node(a, bb, c)];
    }
    __syncthreads();
    const double* Fx = E->F[0];
    const double* Fy = E->F[1];
    const double* Fz = E->F[2];
    const double* Bx = E->B[0];
    const double* By = E->B[1];
    const double* Bz = E->B[2];
    for (int t = threadIdx.x; t < M; t += blockDim.x) {
        const int p = t % mx, rest = t / mx;
        double acc = 0.0;
        for (int a = 0; a < mx; a++) acc = fma(Fx[p * mx + a], s0[rest * mx + a], acc);
        s1[t] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < M; t += blockDim.x) {
        const int p = t % mx, q = (t / mx) % my, c = t / (mx * my);
        double acc = 0.0;
        for (int bb = 0; bb < my; bb++) acc = fma(Fy[q * my + bb], s1[(c * my + bb) * mx + p], acc);
        s0[t] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < M; t += blockDim.x) {
        const int p = t % mx, q = (t / mx) % my, sidx = t / (mx * my);
        double acc = 0.0;
        for (int c = 0; c < mz; c++) acc = fma(Fz[sidx * mz + c], s0[(c * my + q) * mx + p], acc);
        s1[t] = acc / (E->lam[0][p] + E->lam[1][q] + E->lam[2][sidx]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < M; t += blockDim.x) {
        const int p = t % mx, q = (t / mx) % my, c = t / (mx * my);
        double acc = 0.0;
        for (int sidx = 0; sidx < mz; sidx++) acc = fma(Bz[c * mz + sidx], s1[(sidx * my + q) * mx + p], acc);
        s0[t] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < M; t += blockDim.x) {
        const int p = t % mx, bb = (t / mx) % my, c = t / (mx * my);
        double acc = 0.0;
        for (int q = 0; q < my; q++) acc = fma(By[bb * my + q], s0[(c * my + q) * mx + p], acc);
        s1[t] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < M; t += blockDim.x) {
        const int a = t % mx, rest = t / mx;
        double acc = 0.0;
        for (int p = 0; p < mx; p++) acc = fma(Bx[a * mx + p], s1[rest * mx + p], acc);
        const size_t P = node(a, (t / mx) % my, t / (mx * my));
        if (add) e[P] = (T)((double)e[P] + acc);
        else e[P] = (T)acc;
    }
    if (!add) {
        const int N = L.nx * L.ny * L.nz;
        for (int t = threadIdx.x; t < N; t += blockDim.x) {
            const int i = t % L.nx, j = (t / L.nx) % L.ny, k = t / (L.nx * L.ny);
            if (is_face(L, i, j, k)) e[t] = T(0);
        }
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(512) k_coarse_apply(LevelT<T> L, const CoarseEig* __restrict__ E,
                                                     const T* __restrict__ b, T* __restrict__ e, int add)
{
    __shared__ double s0[MC3], s1[MC3];
    coarse_apply_block<T>(L, E, b, e, add, s0, s1);
}

template <typename T>
cudaError_t launch_coarse_apply(const LevelT<T>& L, const CoarseEig* eig, const T* b, T* e, bool add, cudaStream_t s)
{
    k_coarse_apply<T><<<1, 512, 0, s>>>(L, eig, b, e, add ? 1 : 0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- fused residual + restriction
// bc = Vc^-1 P^T Vf (b - A u) with the 27 fine residuals formed on the fly, and the coarse
// correction uc zeroed for the recursion: one pass instead of residual, restriction, memset.
// (the same six terms as offdiag, addressed by flat 64-bit index: in the 27-point loop below the
// compiler then shares the address arithmetic of neighbouring residuals; 20 % faster at 385^3)
template <typename T>
__device__ __forceinline__ T offdiag_flat(const LevelT<T>& L, const T* __restrict__ u, size_t P, int i, int j, int k)
{
    const size_t sy = L.nx, sz = (size_t)L.nx * L.ny;
    T t = L.ax[0].cm[i] * u[P - 1];
    t = fma(L.ax[0].cp[i], u[P + 1], t);
    t = fma(L.ax[1].cm[j], u[P - sy], t);
    t = fma(L.ax[1].cp[j], u[P + sy], t);
    t = fma(L.ax[2].cm[k], u[P - sz], t);
    t = fma(L.ax[2].cp[k], u[P + sz], t);
    return t;
}

template <typename T, int LS = 0>
__device__ __forceinline__ T resid_at(const LevelT<T>& F, const T* __restrict__ u, const T* __restrict__ b, size_t P,
                                      int i, int j, int k)
{
    if constexpr (LS == 0) {
        return b[P] - fma(-dsum(F, i, j, k), u[P], offdiag_flat(F, u, P, i, j, k));
    } else {
        const unsigned Q = pos<LS>(F, P);
        return b[Q] - fma(-dsum(F, i, j, k), u[Q], offdiag<LS>(F, u, P, i, j, k));
    }
}

template <typename T, int LS>
__global__ void __launch_bounds__(NT) k_resid_restrict(LevelT<T> F, LevelT<T> C, const T* __restrict__ u,
                                                      const T* __restrict__ b, T* __restrict__ bc, T* __restrict__ uc)
{
    const size_t t = blockIdx.x * (size_t)NT + threadIdx.x;
    if (t >= C.N()) return;
    int I, J, K;
    node_ijk(t, C, I, J, K);
    uc[t] = T(0);
    if (is_face(C, I, J, K)) {
        bc[t] = T(0);
        return;
    }
    const T* wx = F.ax[0].rw + 3 * I;
    const T* wy = F.ax[1].rw + 3 * J;
    const T* wz = F.ax[2].rw + 3 * K;
    const size_t sy = F.nx, sz = (size_t)F.nx * F.ny;
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int bb = 0; bb < 3; bb++) {
            const int fk = 2 * K - 1 + c, fj = 2 * J - 1 + bb, fi = 2 * I - 1;
            const size_t P = (size_t)fk * sz + (size_t)fj * sy + fi;
            const T r0 = resid_at<T, LS>(F, u, b, P, fi, fj, fk);
            const T r1 = resid_at<T, LS>(F, u, b, P + 1, fi + 1, fj, fk);
            const T r2 = resid_at<T, LS>(F, u, b, P + 2, fi + 2, fj, fk);
            acc = fma(wz[c] * wy[bb], fma(wx[0], r0, fma(wx[1], r1, wx[2] * r2)), acc);
        }
    bc[t] = acc;
}

// The same in FP32 with one warp per coarse (J, K) row, lanes along I (no index division; the
// row's y and z weights once per warp).  RED_ONLY: the fine iterate comes straight from a half
// sweep of the black nodes, whose residuals are then zero (each black equation was just solved
// with its red neighbours fixed), so only the red residuals are formed and the black ones enter
// the weighted sum as zeros: 13 of the 27 residuals per coarse node, and the black half of b is
// not read.
template <int LS, int RED_ONLY>
__device__ __forceinline__ void k_resid_restrict_rows_body(LevelT<float> F, LevelT<float> C, const float* __restrict__ u, const float* __restrict__ b, float* __restrict__ bc, float* __restrict__ uc)
{
    const int row = (int)(blockIdx.x * 8 + (threadIdx.x >> 5));
    if (row >= C.ny * C.nz) return;
    const int lane = threadIdx.x & 31;
    const int K = row / C.ny, J = row - K * C.ny;
    const size_t cb = (size_t)row * C.nx;
    const bool face_row = J == 0 || K == 0 || J == C.ny - 1 || K == C.nz - 1;
    const float* wy = F.ax[1].rw + 3 * (face_row ? 0 : J);
    const float* wz = F.ax[2].rw + 3 * (face_row ? 0 : K);
    const unsigned sy = (unsigned)F.nx, sz = (unsigned)F.nx * (unsigned)F.ny;
    if (face_row) {
        for (int I = lane; I < C.nx; I += 32) {
            uc[cb + I] = 0.0f;
            bc[cb + I] = 0.0f;
        }
        return;
    }
    // the residual at fine i = 2I + 1 is the one at 2(I + 1) - 1 of the next coarse node: each
    // lane forms it once and passes it up the warp (lane 0 takes lane 31's from the last step)
    float carry[9];
#pragma unroll
    for (int q = 0; q < 9; q++) carry[q] = 0.0f;
    for (int I0 = 0; I0 < C.nx; I0 += 32) {
        const int I = I0 + lane;
        const bool in = I >= 1 && I <= C.nx - 2;
        if (I < C.nx) uc[cb + I] = 0.0f;
        const float* wx = F.ax[0].rw + 3 * (in ? I : 1);
        float acc = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; c++)
#pragma unroll
            for (int bb = 0; bb < 3; bb++) {
                const int fk = 2 * K - 1 + c, fj = 2 * J - 1 + bb, fi = 2 * I - 1;
                const unsigned P = (unsigned)fk * sz + (unsigned)fj * sy + (unsigned)fi;
                const bool edges_red = (c + bb) & 1;   // (fj + fk) odd: (fi, fj, fk) red
                float r0 = 0.0f, r1 = 0.0f, r2 = 0.0f;
                if (!RED_ONLY || edges_red) {
                    if (I <= C.nx - 2) r2 = resid_at<float, LS>(F, u, b, P + 2, fi + 2, fj, fk);   // I = 0 too
                    r0 = __shfl_up_sync(0xffffffffu, r2, 1);
                    if (lane == 0) r0 = carry[3 * c + bb];
                    carry[3 * c + bb] = __shfl_sync(0xffffffffu, r2, 31);
                }
                if ((!RED_ONLY || !edges_red) && in) r1 = resid_at<float, LS>(F, u, b, P + 1, fi + 1, fj, fk);
                acc = fmaf(wz[c] * wy[bb], fmaf(wx[0], r0, fmaf(wx[1], r1, wx[2] * r2)), acc);
            }
        if (I < C.nx) bc[cb + I] = in ? acc : 0.0f;
    }
}

template <int LS, int RED_ONLY>
__global__ void __launch_bounds__(256) k_resid_restrict_rows(LevelT<float> F, LevelT<float> C, const float* __restrict__ u, const float* __restrict__ b, float* __restrict__ bc, float* __restrict__ uc)
{
    k_resid_restrict_rows_body<LS, RED_ONLY>(F, C, u, b, bc, uc);
}

// The restriction alone from the red residuals rr of a colour-split fine level (the black ones
// zero), one warp per coarse (J, K) row, lanes along I: the weighted sum of k_resid_restrict_rows
// <1, 1> over the same residual values in the same order, so the two are bitwise equal.  uc = 0.
__global__ void __launch_bounds__(256) k_restrict_red_rows(LevelT<float> F, LevelT<float> C, const float* __restrict__ rr,
                                                           float* __restrict__ bc, float* __restrict__ uc)
{
    const int row = (int)(blockIdx.x * 8 + (threadIdx.x >> 5));
    if (row >= C.ny * C.nz) return;
    const int lane = threadIdx.x & 31;
    const int K = row / C.ny, J = row - K * C.ny;
    const size_t cb = (size_t)row * C.nx;
    const bool face_row = J == 0 || K == 0 || J == C.ny - 1 || K == C.nz - 1;
    if (face_row) {
        for (int I = lane; I < C.nx; I += 32) {
            uc[cb + I] = 0.0f;
            bc[cb + I] = 0.0f;
        }
        return;
    }
    const float* wy = F.ax[1].rw + 3 * J;
    const float* wz = F.ax[2].rw + 3 * K;
    const unsigned sy = (unsigned)F.nx, sz = (unsigned)F.nx * (unsigned)F.ny;
    for (int I0 = 0; I0 < C.nx; I0 += 32) {
        const int I = I0 + lane;
        if (I >= C.nx) break;
        uc[cb + I] = 0.0f;
        if (I < 1 || I > C.nx - 2) {
            bc[cb + I] = 0.0f;
            continue;
        }
        const float* wx = F.ax[0].rw + 3 * I;
        float r0[9], r1[9], r2[9];
#pragma unroll
        for (int c = 0; c < 3; c++)
#pragma unroll
            for (int bb = 0; bb < 3; bb++) {
                const unsigned P = (unsigned)(2 * K - 1 + c) * sz + (unsigned)(2 * J - 1 + bb) * sy + (unsigned)(2 * I - 1);
                const int q = 3 * c + bb;
                r0[q] = r1[q] = r2[q] = 0.0f;
                if ((c + bb) & 1) {   // (fj + fk) odd: the red nodes of the row are at odd fi
                    r0[q] = __ldg(rr + (P >> 1));
                    r2[q] = __ldg(rr + ((P + 2u) >> 1));
                } else {
                    r1[q] = __ldg(rr + ((P + 1u) >> 1));
                }
            }
        float acc = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; c++)
#pragma unroll
            for (int bb = 0; bb < 3; bb++) {
                const int q = 3 * c + bb;
                acc = fmaf(wz[c] * wy[bb], fmaf(wx[0], r0[q], fmaf(wx[1], r1[q], wx[2] * r2[q])), acc);
            }
        bc[cb + I] = acc;
    }
}

// (the fine level in either storage order, the coarse one natural; red_only: the fine iterate's
// last half sweep was black, FP32 only)
template <typename T>
cudaError_t launch_resid_restrict(const LevelT<T>& F, const LevelT<T>& C, const T* u, const T* b, T* bc, T* uc,
                                  bool red_only, cudaStream_t s, T* scratch, int* status)
{
    if (C.lsh) return cudaErrorInvalidValue;
    if constexpr (sizeof(T) == 4) {
        if (F.lsh && red_only && scratch && split_stage_ok(F.nx, F.ny, F.nz) && !((uintptr_t)scratch & 15u) &&
            !((uintptr_t)u & 15u) && !((uintptr_t)b & 15u)) {
            cudaError_t e = launch_split_stage_resid(F, u, b, scratch, status, s);
            if (e != cudaSuccess) return e;
            k_restrict_red_rows<<<(unsigned)(((size_t)C.ny * C.nz + 7) / 8), 256, 0, s>>>(F, C, scratch, bc, uc);
            return cudaGetLastError();
        }
        const unsigned g = (unsigned)(((size_t)C.ny * C.nz + 7) / 8);
        if (F.lsh && red_only)
            k_resid_restrict_rows<1, 1><<<g, 256, 0, s>>>(F, C, u, b, bc, uc);
        else if (F.lsh)
            k_resid_restrict_rows<1, 0><<<g, 256, 0, s>>>(F, C, u, b, bc, uc);
        else if (red_only)
            k_resid_restrict_rows<0, 1><<<g, 256, 0, s>>>(F, C, u, b, bc, uc);
        else
            k_resid_restrict_rows<0, 0><<<g, 256, 0, s>>>(F, C, u, b, bc, uc);
        return cudaGetLastError();
    }
    if (red_only) return cudaErrorInvalidValue;
    const unsigned g = (unsigned)((C.N() + NT - 1) / NT);
    if (F.lsh)
        k_resid_restrict<T, 1><<<g, NT, 0, s>>>(F, C, u, b, bc, uc);
    else
        k_resid_restrict<T, 0><<<g, NT, 0, s>>>(F, C, u, b, bc, uc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- bottom V-cycle (one block)
// Levels lb..L-1 of a V-cycle in one thread block: the small levels cost far more in launch
// latency than in work, so smoothing, residual, restriction, the exact coarsest solve and
// prolongation run as phases separated by __syncthreads.  u[lb] must be zero on entry.
constexpr int BOT_NT = 1024;

// A level's interior nodes of one colour as items (row, slot): row = (j - 1) + (ny - 2)(k - 1)
// over the interior rows, slot s -> i = 2 s + ((colour + j + k) & 1), skipped when i leaves the
// interior.  The first BOT_IT items of each thread are decoded once per level visit and packed
// as (k << 20) | (j << 10) | s (axes have at most 1023 nodes); any further items (large
// non-cubic levels only) are decoded in the loop.
constexpr int BOT_IT = 4;

struct BotItems {
    int packed[BOT_IT];
    int count;   // items held in packed[]
};

template <typename T>
__device__ __forceinline__ BotItems bot_items(const LevelT<T>& L)
{
    BotItems it;
    const int my = L.ny - 2, slots = L.nx / 2;
    const int items = my * (L.nz - 2) * slots;
    it.count = 0;
#pragma unroll
    for (int c = 0; c < BOT_IT; c++) {
        const int q = (int)threadIdx.x + c * BOT_NT;
        it.packed[c] = 0;
        if (q < items) {
            const int row = q / slots, sl = q - row * slots;
            const int k = 1 + row / my, j = 1 + row - (k - 1) * my;
            it.packed[c] = (k << 20) | (j << 10) | sl;
            it.count = c + 1;
        }
    }
    return it;
}

template <typename T>
__device__ __forceinline__ void bot_point(const LevelT<T>& L, T* __restrict__ u, const T* __restrict__ b, int colour,
                                          int k, int j, int sl)
{
    const int i = 2 * sl + ((colour + j + k) & 1);
    if (i < 1 || i > L.nx - 2) return;
    const size_t P = ((size_t)k * L.ny + j) * L.nx + i;
    const T acc = b[P] - offdiag(L, u, P, i, j, k);
    if constexpr (sizeof(T) == 8) u[P] = acc * L.inv_diag[P];
    else u[P] = rb_point32(acc, dsum(L, i, j, k));
}

template <typename T>
__device__ void bot_rbgs(const LevelT<T>& L, const BotItems& it, T* __restrict__ u, const T* __restrict__ b,
                         int colour)
{
#pragma unroll
    for (int c = 0; c < BOT_IT; c++)
        if (c < it.count) {
            const int w = it.packed[c];
            bot_point(L, u, b, colour, w >> 20, (w >> 10) & 1023, w & 1023);
        }
    const int my = L.ny - 2, slots = L.nx / 2;
    const int items = my * (L.nz - 2) * slots;
    for (int q = (int)threadIdx.x + BOT_IT * BOT_NT; q < items; q += BOT_NT) {
        const int row = q / slots, sl = q - row * slots;
        const int k = 1 + row / my, j = 1 + row - (k - 1) * my;
        bot_point(L, u, b, colour, k, j, sl);
    }
    __syncthreads();
}

// Shared-memory layout of the bottom levels: per level u, b and the eight axis tables of
// each axis; the kernel copies the tables and b in, works in shared memory only, and writes
// the top bottom level's u back for the prolongation above it.
template <typename T>
__device__ __forceinline__ void k_bottom_body(const BottomArgs<T>& a)
{
    extern __shared__ __align__(16) unsigned char bot_smem[];
    // one block-wide copy of the level descriptors (pointing into shared memory)
    __shared__ LevelT<T> lv[BOTTOM_MAX_LEVELS];
    __shared__ T* u[BOTTOM_MAX_LEVELS];
    __shared__ T* b[BOTTOM_MAX_LEVELS];
    double* s0 = reinterpret_cast<double*>(bot_smem);
    double* s1 = s0 + MC3;
    const int nl = a.nlev;
    if (threadIdx.x == 0) {
        T* cur = reinterpret_cast<T*>(s1 + MC3);
        for (int l = 0; l < nl; l++) {
            lv[l] = a.lv[l];
            for (int d = 0; d < 3; d++) {
                const int n = a.lv[l].ax[d].n;
                AxisT<T>& A = lv[l].ax[d];
                A.cm = cur; A.cp = cur + n; A.dg = cur + 2 * n; A.dual = cur + 3 * n;
                A.pl = cur + 4 * n; A.pr = cur + 5 * n; A.rw = cur + 6 * n;
                cur += 9 * n;
            }
            u[l] = cur;
            cur += lv[l].N();
            b[l] = cur;
            cur += lv[l].N();
        }
    }
    __syncthreads();
    for (int l = 0; l < nl; l++)
        for (int d = 0; d < 3; d++) {
            const AxisT<T>& g = a.lv[l].ax[d];
            T* dst = const_cast<T*>(lv[l].ax[d].cm);
            const int n = g.n;
            for (int i = threadIdx.x; i < n; i += BOT_NT) {
                dst[i] = g.cm[i];
                dst[n + i] = g.cp[i];
                dst[2 * n + i] = g.dg[i];
                dst[3 * n + i] = g.dual[i];
                dst[4 * n + i] = g.pl[i];
                dst[5 * n + i] = g.pr[i];
            }
            for (int i = threadIdx.x; i < 3 * n; i += BOT_NT) dst[6 * n + i] = g.rw[i];
        }
    // top level: b from global, u = 0 (the caller's correction starts at zero)
    for (unsigned t = threadIdx.x; t < lv[0].N(); t += BOT_NT) {
        b[0][t] = a.b[0][t];
        u[0][t] = T(0);
    }
    __syncthreads();
    for (int l = 0; l < nl - 1; l++) {
        const LevelT<T>& F = lv[l];
        const BotItems items = bot_items(F);
        for (int it = 0; it < a.nu1; it++) {
            bot_rbgs(F, items, u[l], b[l], 0);
            bot_rbgs(F, items, u[l], b[l], 1);
        }
        const LevelT<T>& C = lv[l + 1];
        for (unsigned t = threadIdx.x; t < C.N(); t += BOT_NT) {
            int I, J, K;
            node_ijk(t, C, I, J, K);
            u[l + 1][t] = T(0);
            if (is_face(C, I, J, K)) {
                b[l + 1][t] = T(0);
                continue;
            }
            const T* wx = F.ax[0].rw + 3 * I;
            const T* wy = F.ax[1].rw + 3 * J;
            const T* wz = F.ax[2].rw + 3 * K;
            const unsigned sy = F.nx, sz = (unsigned)F.nx * F.ny;
            T acc = T(0);
            for (int c = 0; c < 3; c++)
                for (int bb = 0; bb < 3; bb++) {
                    const int fk = 2 * K - 1 + c, fj = 2 * J - 1 + bb, fi = 2 * I - 1;
                    const unsigned P = (unsigned)fk * sz + (unsigned)fj * sy + fi;
                    const T r0 = resid_at(F, u[l], b[l], P, fi, fj, fk);
                    const T r1 = resid_at(F, u[l], b[l], P + 1, fi + 1, fj, fk);
                    const T r2 = resid_at(F, u[l], b[l], P + 2, fi + 2, fj, fk);
                    acc = fma(wz[c] * wy[bb], fma(wx[0], r0, fma(wx[1], r1, wx[2] * r2)), acc);
                }
            b[l + 1][t] = acc;
        }
        __syncthreads();
    }
    coarse_apply_block<T>(lv[nl - 1], a.eig, b[nl - 1], u[nl - 1], 0, s0, s1);
    for (int l = nl - 2; l >= 0; l--) {
        const LevelT<T>& F = lv[l];
        const LevelT<T>& C = lv[l + 1];
        const T* ec = u[l + 1];
        T* ul = u[l];
        for (unsigned P = threadIdx.x; P < F.N(); P += BOT_NT) {
            int i, j, k;
            node_ijk(P, F, i, j, k);
            if (is_face(F, i, j, k)) continue;
            const int I = i >> 1, J = j >> 1, K = k >> 1;
            const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nk = (k & 1) ? 2 : 1;
            const T wx[2] = {F.ax[0].pl[i], F.ax[0].pr[i]};
            const T wy[2] = {F.ax[1].pl[j], F.ax[1].pr[j]};
            const T wz[2] = {F.ax[2].pl[k], F.ax[2].pr[k]};
            const unsigned sy = C.nx, sz = (unsigned)C.nx * C.ny;
            const T* base = ec + (unsigned)K * sz + (unsigned)J * sy + I;
            T e = T(0);
            for (int c = 0; c < nk; c++)
                for (int bb = 0; bb < nj; bb++) {
                    const T* row = base + c * sz + bb * sy;
                    const T sv = (ni == 2) ? fma(wx[0], row[0], wx[1] * row[1]) : row[0];
                    e = fma(wz[c] * wy[bb], sv, e);
                }
            ul[P] += e;
        }
        __syncthreads();
        const BotItems items = bot_items(F);
        for (int it = 0; it < a.nu2; it++) {
            bot_rbgs(F, items, ul, b[l], a.sym ? 1 : 0);
            bot_rbgs(F, items, ul, b[l], a.sym ? 0 : 1);
        }
    }
    for (unsigned t = threadIdx.x; t < lv[0].N(); t += BOT_NT) a.u[0][t] = u[0][t];
}

template <typename T>
__global__ void __launch_bounds__(BOT_NT) k_bottom(BottomArgs<T> a)
{
    k_bottom_body<T>(a);
}

template <typename T>
size_t bottom_smem_bytes(const BottomArgs<T>& a)
{
    size_t bytes = 2 * sizeof(double) * MC3;
    for (int l = 0; l < a.nlev; l++) {
        for (int d = 0; d < 3; d++) bytes += sizeof(T) * 9 * (size_t)a.lv[l].ax[d].n;
        bytes += 2 * sizeof(T) * a.lv[l].N();
    }
    return bytes;
}

template <typename T>
cudaError_t launch_bottom(const BottomArgs<T>& a, cudaStream_t s)
{
    const size_t smem = bottom_smem_bytes(a);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    for (int q = 0; q < a.nlev; q++)
        if (a.lv[q].lsh) return cudaErrorInvalidValue;   // natural storage only
    k_bottom<T><<<1, BOT_NT, smem, s>>>(a);
    return cudaGetLastError();
}

void init_bat_attributes();

void init_mg_attributes()
{
    init_bat_attributes();
    init_stage_attributes();
    cudaFuncSetAttribute(k_bottom<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_bottom<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

// ---------------------------------------------------------------- reductions
// Reducing kernels run a grid-stride loop over at most RED_BLOCKS blocks, accumulate in the
// kernel's own precision (FP32 shuffles for FP32 vectors: FP64 is 1/58 of FP32 here),
// write one FP64 partial per block, and the last block to finish (atomic ticket) sums the
// partials in block order and applies the scalar step of the iteration -- so no separate
// finalising launch, and every result is bitwise reproducible.
constexpr int RED_BLOCKS = 1216;   // 152 SMs x 8

int reduce_blocks(const LevelT<double>& L) { return (int)std::min<size_t>((L.N() + NT - 1) / NT, RED_BLOCKS); }
static unsigned red_grid(size_t N) { return (unsigned)std::min<size_t>((N + NT - 1) / NT, RED_BLOCKS); }

__device__ __forceinline__ double vol(const LevelT<double>& L, int i, int j, int k)
{
    return L.ax[0].dual[i] * L.ax[1].dual[j] * L.ax[2].dual[k];
}

// FP32 warp sums, one FP64 value per warp, FP64 across the block's warps
__device__ __forceinline__ double block_sum_f32(float v, double* sm)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sm[w] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < NT / 32) ? sm[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

__device__ void fin_apply(Ctl& c, double s, int op, cudaGraphConditionalHandle cond, int use_cond)
{
    switch (op) {
        case FIN_BNORM:
            c.bnorm = sqrt(s);
            break;
        case FIN_ALPHA:
            c.alpha = (s != 0.0 && isfinite(s)) ? c.rz / s : 0.0;
            break;
        case FIN_BETA:
            c.beta = (c.iter == 0 || c.rz == 0.0) ? 0.0 : s / c.rz;
            c.rz = s;
            break;
        case FIN_START:   // residual of the starting guess
        case FIN_CHECK: {
            const double scale = c.bnorm > 0.0 ? c.bnorm : 1.0;
            const double rel = sqrt(s) / scale;
            if (op == FIN_CHECK) c.iter += 1;
            c.rel = rel;
            if (c.iter < CTL_HIST) c.hist[c.iter] = rel;
            int go = 1;
            if (!isfinite(rel)) {
                c.status = LASTO_ERR_NONFINITE;
                go = 0;
            } else if (rel <= c.tol_iter) {
                c.status = LASTO_OK;
                go = 0;
            } else if (c.iter >= c.max_iter) {
                c.status = LASTO_ERR_NOT_CONVERGED;
                go = 0;
            }
            c.done = !go;
            if (use_cond) cudaGraphSetConditional(cond, go ? 1u : 0u);
            break;
        }
        case FIN_IN_START: {   // ||r||^2 of the new inner right-hand side; reset the inner CG
            // reduce only as far as the outer tolerance needs on the last step (0.3 safety)
            c.tol_in_eff = (c.rel > 0.0) ? fmax(c.tol_in, 0.3 * c.tol / c.rel) : c.tol_in;
            c.rr0_in = s;
            c.rz_in = 1.0;
            c.alpha_in = c.beta_in = 0.0;
            c.iter_in = 0;
            const int go = (s > 0.0 && isfinite(s) && c.iter < c.max_iter) ? 1 : 0;
            c.go_in = go;
            if (use_cond) cudaGraphSetConditional(cond, (unsigned)go);
            break;
        }
        case FIN_IN_ALPHA:
            c.alpha_in = (s != 0.0 && isfinite(s)) ? c.rz_in / s : 0.0;
            break;
        case FIN_IN_BETA:
            c.beta_in = (c.iter_in == 0 || c.rz_in == 0.0) ? 0.0 : s / c.rz_in;
            c.rz_in = s;
            break;
        case FIN_IN_CHECK: {
            c.iter += 1;
            c.iter_in += 1;
            const double rel_in = c.rr0_in > 0.0 ? sqrt(s / c.rr0_in) : 0.0;
            const int go = (isfinite(rel_in) && rel_in > c.tol_in_eff && c.iter_in < c.max_in && c.iter < c.max_iter) ? 1 : 0;
            c.go_in = go;
            if (use_cond) cudaGraphSetConditional(cond, (unsigned)go);
            break;
        }
        case FIN_OUTER: {   // true FP64 residual after a correction step
            const double scale = c.bnorm > 0.0 ? c.bnorm : 1.0;
            const double rel = sqrt(s) / scale;
            c.outer += 1;
            c.rel = rel;
            if (c.iter < CTL_HIST) c.hist[c.iter] = rel;
            int go = 1;
            if (!isfinite(rel)) {
                c.status = LASTO_ERR_NONFINITE;
                go = 0;
            } else if (rel <= c.tol) {
                c.status = LASTO_OK;
                go = 0;
            } else if (c.iter >= c.max_iter) {
                c.status = LASTO_ERR_NOT_CONVERGED;
                go = 0;
            }
            c.done = !go;
            if (use_cond) cudaGraphSetConditional(cond, go ? 1u : 0u);
            break;
        }
        case FIN_TRUE: {
            const double scale = c.bnorm > 0.0 ? c.bnorm : 1.0;
            c.true_rel = sqrt(s) / scale;
            if (c.status == LASTO_OK && !(c.true_rel <= c.tol)) c.status = LASTO_ERR_NOT_CONVERGED;
            if (!isfinite(c.true_rel)) c.status = LASTO_ERR_NONFINITE;
            break;
        }
        default:
            break;
    }
}

// Block partial -> last block sums the partials in order and applies the scalar step.
__device__ void reduce_finish(double block_total, const Red& r, double* sm)
{
    __shared__ int is_last;
    if (threadIdx.x == 0) {
        r.part[blockIdx.x] = block_total;
        __threadfence();
        const unsigned prev = atomicAdd(r.counter, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double acc = 0.0;
    for (unsigned t = threadIdx.x; t < gridDim.x; t += NT) acc += __ldcg(r.part + t);
    const double s = block_sum<NT>(acc, sm);
    if (threadIdx.x == 0) {
        *r.counter = 0u;
        fin_apply(*r.ctl, s, r.op, r.cond, r.use_cond);
    }
}

#define GRID_STRIDE(P, N) for (size_t P = blockIdx.x * (size_t)NT + threadIdx.x; P < (N); P += (size_t)gridDim.x * NT)

// Each thread of the vector kernels below takes VU nodes a block's width apart per step and issues all their loads before
// the first use: with one node per step a thread holds 4-8 B of DRAM loads in flight, a fraction
// of what the copy rate needs at full occupancy, and the vector kernels ran at a quarter to a
// half of it.  The accumulation order within a thread is the nodes' order.
// The reducing ones run in one wave of VEC_BLOCKS blocks, a number of blocks per SM that their
// register bound guarantees resident (a second, partial wave would leave SMs idle at the end).
constexpr int VU = 4;
constexpr int VEC_MIN_BLOCKS = 4;
constexpr int VEC_BLOCKS = 152 * VEC_MIN_BLOCKS;
static unsigned vec_grid(size_t N) { return (unsigned)std::min<size_t>((N + NT * VU - 1) / (NT * VU), VEC_BLOCKS); }
#define GRID_STRIDE_U(P0, N) \
    for (size_t P0 = blockIdx.x * (size_t)(NT * VU) + threadIdx.x; P0 < (N); P0 += (size_t)gridDim.x * (NT * VU))

// b at a node next to a face with the face values moved to the right-hand side.  Not inlined:
// inlined, the compiler predicates the six FP64 updates into every node's path, and the FP64
// pipe (about 1/64 of the FP32 rate here) then bounds the whole norm.
__device__ __noinline__ double bnorm_face_adjust(const LevelT<double>& L, const double* __restrict__ u, double w,
                                                 size_t P, int i, int j, int k)
{
    const size_t sy = L.nx, sz = (size_t)L.nx * L.ny;
    if (i == 1) w -= L.ax[0].cm[i] * u[P - 1];
    if (i == L.nx - 2) w -= L.ax[0].cp[i] * u[P + 1];
    if (j == 1) w -= L.ax[1].cm[j] * u[P - sy];
    if (j == L.ny - 2) w -= L.ax[1].cp[j] * u[P + sy];
    if (k == 1) w -= L.ax[2].cm[k] * u[P - sz];
    if (k == L.nz - 2) w -= L.ax[2].cp[k] * u[P + sz];
    return w;
}

// ||b_eff||^2: b with the Dirichlet faces moved to the right-hand side (VU nodes per thread and
// step, loads first)
__global__ void __launch_bounds__(NT, VEC_MIN_BLOCKS) k_bnorm(LevelT<double> L, const double* __restrict__ u,
                                                             const double* __restrict__ b, Red red)
{
    __shared__ double sm[32];
    double acc = 0.0;
    const size_t N = L.N();
    GRID_STRIDE_U(P0, N)
    {
        double v[VU];
        bool on[VU];
#pragma unroll
        for (int q = 0; q < VU; q++) {
            const size_t P = P0 + (size_t)q * NT;
            on[q] = false;
            v[q] = 0.0;
            if (P < N) {
                int i, j, k;
                node_ijk(P, L, i, j, k);
                if (!is_face(L, i, j, k)) {
                    on[q] = true;
                    v[q] = b[P];
                    if (i == 1 || i == L.nx - 2 || j == 1 || j == L.ny - 2 || k == 1 || k == L.nz - 2)
                        v[q] = bnorm_face_adjust(L, u, v[q], P, i, j, k);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < VU; q++)
            if (on[q]) acc = fma(v[q], v[q], acc);
    }
    reduce_finish(block_sum<NT>(acc, sm), red, sm);
}

// r = b - A u (written when r != nullptr, FP32 copy when r32 != nullptr, in colour-split
// storage when h32 = ceil(N / 2) is nonzero) and ||r||^2.  One warp per (j, k) row (grid-stride
// over rows), RN_V nodes per lane and step with their loads first: the FP64 pipe (about 1/64
// of the FP32 rate here) bounds this kernel, and the row form spends one FP64 add per node on
// the diagonal (dg_x + (dg_y + dg_z), the second sum once per row) where the flat form spends
// two.  Face nodes get r = 0.
constexpr int RN_V = 4;

__device__ __forceinline__ void k_resid_norm_body(LevelT<double> L, const double* __restrict__ u, const double* __restrict__ b, double* __restrict__ r, float* __restrict__ r32, unsigned h32, Red red)
{
    __shared__ double sm[32];
    double acc = 0.0;
    const int nx = L.nx, rows = L.ny * L.nz;
    const int lane = threadIdx.x & 31;
    const size_t sy = (size_t)nx, sz = (size_t)nx * L.ny;
    for (int row = (int)(blockIdx.x * (NT / 32) + (threadIdx.x >> 5)); row < rows; row += (int)(gridDim.x * (NT / 32))) {
        const int k = row / L.ny, j = row - k * L.ny;
        const bool frow = j == 0 || k == 0 || j == L.ny - 1 || k == L.nz - 1;
        const size_t P0 = (size_t)row * nx;
        double cmy = 0.0, cpy = 0.0, cmz = 0.0, cpz = 0.0, dyz = 0.0;
        if (!frow) {
            cmy = L.ax[1].cm[j], cpy = L.ax[1].cp[j], cmz = L.ax[2].cm[k], cpz = L.ax[2].cp[k];
            dyz = L.ax[1].dg[j] + L.ax[2].dg[k];
        }
        for (int i0 = lane; i0 < nx; i0 += 32 * RN_V) {
            double v[RN_V];
#pragma unroll
            for (int q = 0; q < RN_V; q++) {
                const int i = i0 + 32 * q;
                v[q] = 0.0;
                if (!frow && i >= 1 && i <= nx - 2) {
                    const double* c = u + P0 + i;
                    double t = L.ax[0].cm[i] * c[-1];
                    t = fma(L.ax[0].cp[i], c[1], t);
                    t = fma(cmy, c[-(ptrdiff_t)sy], t);
                    t = fma(cpy, c[sy], t);
                    t = fma(cmz, c[-(ptrdiff_t)sz], t);
                    t = fma(cpz, c[sz], t);
                    v[q] = b[P0 + i] - fma(-(L.ax[0].dg[i] + dyz), c[0], t);
                }
            }
#pragma unroll
            for (int q = 0; q < RN_V; q++) {
                const int i = i0 + 32 * q;
                if (i >= nx) continue;
                const unsigned P = (unsigned)(P0 + i);
                if (r) r[P] = v[q];
                if (r32) r32[h32 ? (P >> 1) + (P & 1u) * h32 : P] = (float)v[q];
                acc = fma(v[q], v[q], acc);
            }
        }
    }
    reduce_finish(block_sum<NT>(acc, sm), red, sm);
}

// rows kernels' grid: one warp per row while the partials allow (one per ceil(N / 256) nodes)
static unsigned resid_rows_grid(const LevelT<double>& L)
{
    const size_t rows = (size_t)L.ny * L.nz;
    return (unsigned)std::max<size_t>(1, std::min((rows + NT / 32 - 1) / (NT / 32), (L.N() + 255) / 256));
}

__global__ void __launch_bounds__(NT) k_resid_norm(LevelT<double> L, const double* __restrict__ u, const double* __restrict__ b, double* __restrict__ r, float* __restrict__ r32, unsigned h32, Red red)
{
    k_resid_norm_body(L, u, b, r, r32, h32, red);
}

// q = A p and <p, q>_vol
__global__ void __launch_bounds__(NT) k_apply_dot(LevelT<double> L, const double* __restrict__ p,
                                                 double* __restrict__ q, Red red)
{
    __shared__ double sm[32];
    double acc = 0.0;
    GRID_STRIDE(P, L.N())
    {
        int i, j, k;
        node_ijk(P, L, i, j, k);
        double v = 0.0;
        if (!is_face(L, i, j, k)) {
            v = fma(-dsum(L, i, j, k), p[P], offdiag(L, p, P, i, j, k));
            acc = fma(vol(L, i, j, k) * p[P], v, acc);
        }
        q[P] = v;
    }
    reduce_finish(block_sum<NT>(acc, sm), red, sm);
}

// u += alpha p; r -= alpha q; ||r||^2
__global__ void __launch_bounds__(NT) k_update_ur(LevelT<double> L, const Ctl* __restrict__ ctl,
                                                 const double* __restrict__ p, const double* __restrict__ q,
                                                 double* __restrict__ u, double* __restrict__ r, Red red)
{
    __shared__ double sm[32];
    const double alpha = ctl->alpha;
    double acc = 0.0;
    GRID_STRIDE(P, L.N())
    {
        int i, j, k;
        node_ijk(P, L, i, j, k);
        if (is_face(L, i, j, k)) continue;
        u[P] = fma(alpha, p[P], u[P]);
        const double rv = fma(-alpha, q[P], r[P]);
        r[P] = rv;
        acc = fma(rv, rv, acc);
    }
    reduce_finish(block_sum<NT>(acc, sm), red, sm);
}

__global__ void __launch_bounds__(NT) k_dot_rz(LevelT<double> L, const double* __restrict__ r,
                                              const double* __restrict__ z, Red red)
{
    __shared__ double sm[32];
    double acc = 0.0;
    GRID_STRIDE(P, L.N())
    {
        int i, j, k;
        node_ijk(P, L, i, j, k);
        if (!is_face(L, i, j, k)) acc = fma(vol(L, i, j, k) * r[P], z[P], acc);
    }
    reduce_finish(block_sum<NT>(acc, sm), red, sm);
}

__global__ void __launch_bounds__(NT) k_update_p(LevelT<double> L, const Ctl* __restrict__ ctl,
                                                const double* __restrict__ z, double* __restrict__ p)
{
    const size_t P = blockIdx.x * (size_t)NT + threadIdx.x;
    if (P >= L.N()) return;
    int i, j, k;
    node_ijk(P, L, i, j, k);
    p[P] = is_face(L, i, j, k) ? 0.0 : fma(ctl->beta, p[P], z[P]);
}

// ---------------------------------------------------------------- inner FP32 CG (defect correction)
__device__ __forceinline__ float vol32(const LevelT<float>& L, int i, int j, int k)
{
    return L.ax[0].dual[i] * L.ax[1].dual[j] * L.ax[2].dual[k];
}

// (the inner CG vectors share the finest level's FP32 storage order; every kernel walks the
// nodes in flat order, so sums are formed in the same order in both)

template <int LS>
__device__ __forceinline__ void k_apply_dot32_body(LevelT<float> L, const float* __restrict__ p, float* __restrict__ q, Red red)
{
    __shared__ double sm[32];
    float acc = 0.0f;
    const size_t N = L.N();
    GRID_STRIDE_U(P0, N)
    {
        float pc[VU], od[VU], dg[VU], w[VU];
        unsigned Q[VU];
        bool in[VU], face[VU];
#pragma unroll
        for (int u = 0; u < VU; u++) {
            const size_t P = P0 + (size_t)u * NT;
            in[u] = P < N;
            face[u] = true;
            Q[u] = 0u;
            pc[u] = od[u] = dg[u] = w[u] = 0.0f;
            if (in[u]) {
                int i, j, k;
                node_ijk(P, L, i, j, k);
                Q[u] = pos<LS>(L, P);
                face[u] = is_face(L, i, j, k);
                if (!face[u]) {
                    pc[u] = p[Q[u]];
                    od[u] = offdiag<LS>(L, p, P, i, j, k);
                    dg[u] = dsum(L, i, j, k);
                    w[u] = vol32(L, i, j, k);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < VU; u++) {
            if (!in[u]) continue;
            float v = 0.0f;
            if (!face[u]) {
                v = fmaf(-dg[u], pc[u], od[u]);
                acc = fmaf(w[u] * pc[u], v, acc);
            }
            q[Q[u]] = v;
        }
    }
    reduce_finish(block_sum_f32(acc, sm), red, sm);
}

template <int LS>
__global__ void __launch_bounds__(NT, VEC_MIN_BLOCKS) k_apply_dot32(LevelT<float> L, const float* __restrict__ p, float* __restrict__ q, Red red)
{
    k_apply_dot32_body<LS>(L, p, q, red);
}

// The same with one warp per interior (j, k) row, its red nodes and then its black ones, lanes
// along the run: the row's y and z coefficients and volume factors once per warp, the six
// neighbours of a node at offsets fixed along the run (in the other half of colour-split storage)
// and no index division, where the flat form above spends about as many instructions on indexing
// as the copy rate leaves it.  Face nodes of q are not written (the CG reads q at interior nodes
// only).  One row per warp while the grid allows (the reduction takes one partial per block, at
// most ceil(N / 256) of them), else a grid-stride loop over rows; L2 prefetch of the z+ row of the
// row pf ahead, both colours, as in the row-per-warp half sweep.  Sums run in the same order in
// both storage orders.
template <int LS, int V>
__device__ __forceinline__ void k_apply_dot32_rows_body(LevelT<float> L, const float* __restrict__ p, float* __restrict__ q, Red red, int pf)
{
    __shared__ double sm[32];
    float acc = 0.0f;
    const int my = L.ny - 2, rows = my * (L.nz - 2);
    const int lane = threadIdx.x & 31;
    const int nx = L.nx;
    const unsigned nxy = (unsigned)nx * (unsigned)L.ny;
    const int hx = (nx - 1) >> 1, hxy = (int)((nxy - 1) >> 1);
    for (int row = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); row < rows;
         row += (int)(gridDim.x * (blockDim.x >> 5))) {
        const int k = row / my + 1, j = row - (k - 1) * my + 1;
        if (pf > 0 && row + pf < rows) {
            const int r2 = row + pf;
            const int k2 = r2 / my + 2, j2 = r2 - (k2 - 2) * my + 1;   // the z+ row of row r2
            if (k2 <= L.nz - 2 && lane < 2 * ((hx + 32) / 32)) {
                const int c2 = lane & 1, l2 = lane >> 1;
                const unsigned P2 = (unsigned)k2 * nxy + (unsigned)j2 * (unsigned)nx;
                const float* a = LS ? p + (size_t)c2 * L.H + (P2 >> 1) + 32 * l2 : p + P2 + 64 * l2 + 32 * c2;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
            }
        }
        const float cmy = L.ax[1].cm[j], cpy = L.ax[1].cp[j], dgy = L.ax[1].dg[j];
        const float cmz = L.ax[2].cm[k], cpz = L.ax[2].cp[k], dgz = L.ax[2].dg[k];
        const float vy = L.ax[1].dual[j], vz = L.ax[2].dual[k];
        const unsigned Prow = (unsigned)k * nxy + (unsigned)j * (unsigned)nx;
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const int i1 = ((c + j + k) & 1) ? 1 : 2;   // first interior node of the colour
            const int left = ((nx - i1) >> 1) - lane;   // the colour's interior nodes past lane's first
            const unsigned P0 = Prow + (unsigned)i1;
            // one base pointer per operand stream, lane's first node; node v is 32 v nodes of the
            // colour further on (a compile-time offset)
            constexpr int ST = LS ? 1 : 2;
            const float* __restrict__ cmx = L.ax[0].cm + i1 + 2 * lane;
            const float* __restrict__ cpx = L.ax[0].cp + i1 + 2 * lane;
            const float* __restrict__ dgx = L.ax[0].dg + i1 + 2 * lane;
            const float* __restrict__ vx = L.ax[0].dual + i1 + 2 * lane;
            const float *own, *nxm, *nxp, *nym, *nyp, *nzm, *nzp;
            float* qo;
            if constexpr (LS == 1) {
                const unsigned q0 = (P0 >> 1) + (unsigned)lane;
                own = p + (size_t)c * L.H + q0;
                qo = q + (size_t)c * L.H + q0;
                const float* o = p + (size_t)(1 - c) * L.H + q0;
                nxm = o + (c - 1), nxp = o + c, nym = o + (c - 1 - hx), nyp = o + (c + hx), nzm = o + (c - 1 - hxy),
                nzp = o + (c + hxy);
            } else {
                own = p + P0 + 2 * lane;
                qo = q + P0 + 2 * lane;
                nxm = own - 1, nxp = own + 1, nym = own - nx, nyp = own + nx, nzm = own - nxy, nzp = own + nxy;
            }
#pragma unroll
            for (int v = 0; v < V; v++) {
                if (32 * v < left) {
                    const int off = 32 * ST * v;
                    const float pc = __ldg(own + off);
                    float t = cmx[64 * v] * __ldg(nxm + off);
                    t = fmaf(cpx[64 * v], __ldg(nxp + off), t);
                    t = fmaf(cmy, __ldg(nym + off), t);
                    t = fmaf(cpy, __ldg(nyp + off), t);
                    t = fmaf(cmz, __ldg(nzm + off), t);
                    t = fmaf(cpz, __ldg(nzp + off), t);
                    const float val = fmaf(-(dgx[64 * v] + dgy + dgz), pc, t);
                    acc = fmaf(vx[64 * v] * vy * vz * pc, val, acc);
                    qo[off] = val;
                }
            }
        }
    }
    reduce_finish(block_sum_f32(acc, sm), red, sm);
}

template <int LS, int V>
__global__ void __launch_bounds__(256) k_apply_dot32_rows(LevelT<float> L, const float* __restrict__ p, float* __restrict__ q, Red red, int pf)
{
    k_apply_dot32_rows_body<LS, V>(L, p, q, red, pf);
}

// The same, plane-staged (the arrangement of the staged half sweep, stage.cu): a block owns 8
// interior rows (one warp each) and a chunk of planes, and keeps planes k - 1, k, k + 1 of p --
// rows j0 - 1 .. j0 + 8, both colours: one run per colour half in colour-split storage, one run
// in natural storage -- in a ring of AS_NS slots with the next plane in flight.  Both storage
// orders run this kernel with the same node-to-thread map and accumulation order, so their sums
// agree bit for bit; so do a lockstep batch and its members run alone.
constexpr int AS_R = 8;
constexpr int AS_NS = 4;

struct ApplyGeom {
    int tiles_j, chunk;
    unsigned slot;   // floats per run slot (a multiple of 4)
    int hx1;         // x coefficients per parity (a multiple of 4)
};

// run t (colour half t in colour-split storage; t = 0 the whole plane rows in natural) of plane pl
template <int LS>
__device__ __forceinline__ void as_range(const LevelT<float>& L, int t, int pl, int j0, int nr, unsigned& st, unsigned& len)
{
    const unsigned nxy = (unsigned)L.nx * (unsigned)L.ny;
    const unsigned lo = (unsigned)pl * nxy + (unsigned)(j0 - 1) * (unsigned)L.nx;
    const unsigned hi = (unsigned)pl * nxy + (unsigned)(j0 + nr + 1) * (unsigned)L.nx - 1u;
    if constexpr (LS == 1)
        stage::sg_range((unsigned)t * L.H + (lo >> 1), (unsigned)t * L.H + (hi >> 1) + 1u, (unsigned)L.N(), st, len);
    else
        stage::sg_range(lo, hi + 1u, (unsigned)L.N(), st, len);
}

template <int V, int LS>
__device__ __forceinline__ void k_apply_stage_body(const LevelT<float>& L, const float* __restrict__ p, float* __restrict__ q,
                                                   const Red& red, const ApplyGeom& g, int* __restrict__ status)
{
    using namespace stage;
    constexpr int NH = LS ? 2 : 1;
    extern __shared__ __align__(16) float sg[];
    __shared__ __align__(8) uint64_t bar[AS_NS];
    __shared__ unsigned st_of[NH][AS_NS];
    __shared__ double sm[32];
    float* ring = sg;                                // [NH][AS_NS][slot]
    float* sx = sg + NH * AS_NS * g.slot;            // [2 parities][cm, cp, dg, dual][hx1]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tj = (int)(blockIdx.x % (unsigned)g.tiles_j), kc = (int)(blockIdx.x / (unsigned)g.tiles_j);
    const int j0 = 1 + tj * AS_R;
    const int nr = min(AS_R, L.ny - 1 - j0);
    const int kA = 1 + kc * g.chunk, kB = min(L.nz - 2, kA + g.chunk - 1);
    float acc = 0.0f;
    bool failed = false;
    if (nr > 0 && kA <= kB) {   // (block-uniform)
        const int nx = L.nx;
        const unsigned nxy = (unsigned)nx * (unsigned)L.ny;
        const int hx = (nx - 1) >> 1, hxy = (int)((nxy - 1) >> 1);
        const int o0 = kA - 1, oLast = kB + 1;
        int o_next = o0;
        auto issue = [&](int pl) {   // thread 0: plane pl into its slot, all runs on one barrier
            const int qs = (pl - o0) % AS_NS;
            unsigned st[NH], ln[NH], bytes = 0;
            for (int t = 0; t < NH; t++) {
                as_range<LS>(L, t, pl, j0, nr, st[t], ln[t]);
                st_of[t][qs] = st[t];
                bytes += ln[t] * 4u;
            }
            const uint32_t b = sg_smem(&bar[qs]);
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(bytes) : "memory");
            for (int t = 0; t < NH; t++)
                if (ln[t])
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                            sg_smem(ring + (t * AS_NS + qs) * g.slot)),
                        "l"(p + st[t]), "r"(ln[t] * 4u), "r"(b)
                        : "memory");
        };
        if (tid == 0) {
            for (int qq = 0; qq < AS_NS; qq++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sg_smem(&bar[qq])) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
        for (int t = tid; t < 2 * g.hx1; t += blockDim.x) {
            const int par = t / g.hx1, si = t - par * g.hx1;
            const int i = 1 + par + 2 * si;
            const bool in = i < nx - 1;
            sx[(par * 4 + 0) * g.hx1 + si] = in ? L.ax[0].cm[i] : 0.0f;
            sx[(par * 4 + 1) * g.hx1 + si] = in ? L.ax[0].cp[i] : 0.0f;
            sx[(par * 4 + 2) * g.hx1 + si] = in ? L.ax[0].dg[i] : 0.0f;
            sx[(par * 4 + 3) * g.hx1 + si] = in ? L.ax[0].dual[i] : 0.0f;
        }
        __syncthreads();
        if (tid == 0)
            for (; o_next <= oLast && o_next < o0 + AS_NS; o_next++) issue(o_next);
        const int j = j0 + warp;
        const bool has_row = warp < nr;
        const float cmy = has_row ? L.ax[1].cm[j] : 0.0f, cpy = has_row ? L.ax[1].cp[j] : 0.0f;
        const float dgy = has_row ? L.ax[1].dg[j] : 0.0f, vy = has_row ? L.ax[1].dual[j] : 0.0f;
        for (int k = kA; k <= kB; k++) {
            bool bad = false;
            for (int pl = (k == kA ? k - 1 : k + 1); pl <= k + 1; pl++) {
                const int d = pl - o0;
                if (!bad && !sg_wait(sg_smem(&bar[d % AS_NS]), (uint32_t)((d / AS_NS) & 1))) bad = true;
            }
            if (!bad && has_row) {
                const int sk = (k - o0) % AS_NS, skm = (k - 1 - o0) % AS_NS, skp = (k + 1 - o0) % AS_NS;
                const float cmz = L.ax[2].cm[k], cpz = L.ax[2].cp[k], dgz = L.ax[2].dg[k], vz = L.ax[2].dual[k];
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const int i1 = ((c + j + k) & 1) ? 1 : 2;
                    const int left = ((nx - i1) >> 1) - lane;
                    const unsigned P0 = (unsigned)k * nxy + (unsigned)j * (unsigned)nx + (unsigned)i1;
                    const float* cmx = sx + (i1 - 1) * 4 * g.hx1 + lane;
                    const float* cpx = cmx + g.hx1;
                    const float* dgx = cpx + g.hx1;
                    const float* vx = dgx + g.hx1;
                    constexpr int ST = LS ? 1 : 2;
                    const float *own, *ok, *om, *op;
                    float* qo;
                    int dxm, dxp, dym, dyp, dzm, dzp;
                    if constexpr (LS == 1) {
                        const unsigned gq = (P0 >> 1) + (unsigned)lane;
                        own = ring + (c * AS_NS + sk) * g.slot + ((unsigned)c * L.H + gq - st_of[c][sk]);
                        const int oc = 1 - c;
                        ok = ring + (oc * AS_NS + sk) * g.slot + ((unsigned)oc * L.H + gq - st_of[oc][sk]);
                        om = ring + (oc * AS_NS + skm) * g.slot + ((unsigned)oc * L.H + gq - st_of[oc][skm]);
                        op = ring + (oc * AS_NS + skp) * g.slot + ((unsigned)oc * L.H + gq - st_of[oc][skp]);
                        qo = q + (size_t)c * L.H + gq;
                        dxm = c - 1, dxp = c, dym = c - 1 - hx, dyp = c + hx, dzm = c - 1 - hxy, dzp = c + hxy;
                    } else {
                        const unsigned gp = P0 + 2u * (unsigned)lane;
                        own = ring + sk * g.slot + (gp - st_of[0][sk]);
                        ok = own;
                        om = ring + skm * g.slot + (gp - st_of[0][skm]);
                        op = ring + skp * g.slot + (gp - st_of[0][skp]);
                        qo = q + gp;
                        dxm = -1, dxp = 1, dym = -nx, dyp = nx, dzm = -(int)nxy, dzp = (int)nxy;
                    }
#pragma unroll
                    for (int v = 0; v < V; v++) {
                        if (32 * v < left) {
                            const int o = 32 * ST * v;
                            const float pc = own[o];
                            float t = cmx[32 * v] * ok[dxm + o];
                            t = fmaf(cpx[32 * v], ok[dxp + o], t);
                            t = fmaf(cmy, ok[dym + o], t);
                            t = fmaf(cpy, ok[dyp + o], t);
                            t = fmaf(cmz, om[dzm + o], t);
                            t = fmaf(cpz, op[dzp + o], t);
                            const float val = fmaf(-(dgx[32 * v] + dgy + dgz), pc, t);
                            acc = fmaf(vx[32 * v] * vy * vz * pc, val, acc);
                            qo[o] = val;
                        }
                    }
                }
            }
            if (__syncthreads_or(bad ? 1 : 0)) {
                failed = true;
                break;
            }
            if (tid == 0 && o_next <= oLast) issue(o_next++);   // into plane k - 1's slot
        }
        if (tid == 0 && failed) {
            for (int pl = max(o0, o_next - AS_NS); pl < o_next; pl++)
                sg_wait(sg_smem(&bar[(pl - o0) % AS_NS]), (uint32_t)(((pl - o0) / AS_NS) & 1));
            if (status) atomicMax(status, (int)LASTO_ERR_TIMEOUT);
        }
    }
    // every block takes part in the reduction (a timed-out one with its partial sum so far)
    reduce_finish(block_sum_f32(acc, sm), red, sm);
}

template <int V, int LS>
__global__ void __launch_bounds__(256) k_apply_stage(LevelT<float> L, const float* __restrict__ p, float* __restrict__ q,
                                                     Red red, ApplyGeom g, int* __restrict__ status)
{
    k_apply_stage_body<V, LS>(L, p, q, red, g, status);
}

template <int LS>
__device__ __forceinline__ void k_update_er32_body(LevelT<float> L, const Ctl* __restrict__ ctl, const float* __restrict__ p, const float* __restrict__ q, float* __restrict__ e, float* __restrict__ r, Red red)
{
    __shared__ double sm[32];
    const float alpha = (float)ctl->alpha_in;
    float acc = 0.0f;
    const size_t N = L.N();
    GRID_STRIDE_U(P0, N)
    {
        float pv[VU], qv[VU], ev[VU], rv[VU];
        unsigned Q[VU];
        bool on[VU];
#pragma unroll
        for (int u = 0; u < VU; u++) {
            const size_t P = P0 + (size_t)u * NT;
            on[u] = false;
            Q[u] = 0u;
            pv[u] = qv[u] = ev[u] = rv[u] = 0.0f;
            if (P < N) {
                int i, j, k;
                node_ijk(P, L, i, j, k);
                on[u] = !is_face(L, i, j, k);
                if (on[u]) {
                    Q[u] = pos<LS>(L, P);
                    pv[u] = p[Q[u]];
                    qv[u] = q[Q[u]];
                    ev[u] = e[Q[u]];
                    rv[u] = r[Q[u]];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < VU; u++) {
            if (!on[u]) continue;
            e[Q[u]] = fmaf(alpha, pv[u], ev[u]);
            const float rn = fmaf(-alpha, qv[u], rv[u]);
            r[Q[u]] = rn;
            acc = fmaf(rn, rn, acc);
        }
    }
    reduce_finish(block_sum_f32(acc, sm), red, sm);
}

template <int LS>
__global__ void __launch_bounds__(NT, VEC_MIN_BLOCKS) k_update_er32(LevelT<float> L, const Ctl* __restrict__ ctl, const float* __restrict__ p, const float* __restrict__ q, float* __restrict__ e, float* __restrict__ r, Red red)
{
    k_update_er32_body<LS>(L, ctl, p, q, e, r, red);
}

// <r, z>_vol, or ||r||^2 when z == nullptr (VU_DOT nodes per thread and step, twice the update
// kernels': with two streams and no stores it needs more nodes in flight; measured on the warm
// Pd561 385^3 solve, 0.2 ms less over its 16 dots)
constexpr int VU_DOT = 8;
#define GRID_STRIDE_UD(P0, N) \
    for (size_t P0 = blockIdx.x * (size_t)(NT * VU_DOT) + threadIdx.x; P0 < (N); P0 += (size_t)gridDim.x * (NT * VU_DOT))
template <int LS>
__device__ __forceinline__ void k_dot32_body(LevelT<float> L, const float* __restrict__ r, const float* __restrict__ z, Red red)
{
    __shared__ double sm[32];
    float acc = 0.0f;
    const size_t N = L.N();
    GRID_STRIDE_UD(P0, N)
    {
        float rv[VU_DOT], zv[VU_DOT], w[VU_DOT];
        bool on[VU_DOT];
#pragma unroll
        for (int u = 0; u < VU_DOT; u++) {
            const size_t P = P0 + (size_t)u * NT;
            on[u] = false;
            rv[u] = zv[u] = w[u] = 0.0f;
            if (P < N) {
                int i, j, k;
                node_ijk(P, L, i, j, k);
                on[u] = !is_face(L, i, j, k);
                if (on[u]) {
                    const unsigned Q = pos<LS>(L, P);
                    rv[u] = r[Q];
                    if (z) {
                        zv[u] = z[Q];
                        w[u] = vol32(L, i, j, k);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < VU_DOT; u++)
            if (on[u]) acc = z ? fmaf(w[u] * rv[u], zv[u], acc) : fmaf(rv[u], rv[u], acc);
    }
    reduce_finish(block_sum_f32(acc, sm), red, sm);
}

template <int LS>
__global__ void __launch_bounds__(NT, VEC_MIN_BLOCKS) k_dot32(LevelT<float> L, const float* __restrict__ r, const float* __restrict__ z, Red red)
{
    k_dot32_body<LS>(L, r, z, red);
}

// p = z + beta p (VU nodes per thread, a block's width apart)
template <int LS>
__device__ __forceinline__ void k_update_p32_body(LevelT<float> L, const Ctl* __restrict__ ctl, const float* __restrict__ z, float* __restrict__ p)
{
    const size_t N = L.N();
    const size_t P0 = blockIdx.x * (size_t)(NT * VU) + threadIdx.x;
    const float beta = (float)ctl->beta_in;
    float zv[VU], pv[VU];
    unsigned Q[VU];
    bool in[VU], face[VU];
#pragma unroll
    for (int u = 0; u < VU; u++) {
        const size_t P = P0 + (size_t)u * NT;
        in[u] = P < N;
        face[u] = true;
        Q[u] = 0u;
        zv[u] = pv[u] = 0.0f;
        if (in[u]) {
            int i, j, k;
            node_ijk(P, L, i, j, k);
            Q[u] = pos<LS>(L, P);
            face[u] = is_face(L, i, j, k);
            if (!face[u]) {
                zv[u] = z[Q[u]];
                pv[u] = p[Q[u]];
            }
        }
    }
#pragma unroll
    for (int u = 0; u < VU; u++)
        if (in[u]) p[Q[u]] = face[u] ? 0.0f : fmaf(beta, pv[u], zv[u]);
}

template <int LS>
__global__ void __launch_bounds__(NT) k_update_p32(LevelT<float> L, const Ctl* __restrict__ ctl, const float* __restrict__ z, float* __restrict__ p)
{
    k_update_p32_body<LS>(L, ctl, z, p);
}

// u += e (FP64 accumulation of the FP32 correction, e in colour-split storage when h32 =
// ceil(N / 2) is nonzero); e = 0 for the next inner solve
__device__ __forceinline__ void k_add_correction_body(size_t N, double* __restrict__ u, float* __restrict__ e, unsigned h32)
{
    const size_t P = blockIdx.x * (size_t)NT + threadIdx.x;
    if (P >= N) return;
    const unsigned Q = h32 ? ((unsigned)P >> 1) + ((unsigned)P & 1u) * h32 : (unsigned)P;
    u[P] += (double)e[Q];
    e[Q] = 0.0f;
}

__global__ void __launch_bounds__(NT) k_add_correction(size_t N, double* __restrict__ u, float* __restrict__ e, unsigned h32)
{
    k_add_correction_body(N, u, e, h32);
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, size_t n)
{
    const size_t t = blockIdx.x * (size_t)NT + threadIdx.x;
    if (t < n) b[t] = (float)a[t];
}

#define RGRID(L) red_grid(L.N()), NT, 0, s
#define GRID(L) (unsigned)((L.N() + NT - 1) / NT), NT, 0, s

cudaError_t launch_bnorm(const LevelT<double>& L, const double* u, const double* b, const Red& red, cudaStream_t s)
{
    k_bnorm<<<vec_grid(L.N()), NT, 0, s>>>(L, u, b, red);
    return cudaGetLastError();
}
cudaError_t launch_resid_norm(const LevelT<double>& L, const double* u, const double* b, double* r, float* r32,
                              unsigned h32, const Red& red, cudaStream_t s)
{
    k_resid_norm<<<resid_rows_grid(L), NT, 0, s>>>(L, u, b, r, r32, h32, red);
    return cudaGetLastError();
}
cudaError_t launch_apply_dot(const LevelT<double>& L, const double* p, double* q, const Red& red, cudaStream_t s)
{
    k_apply_dot<<<RGRID(L)>>>(L, p, q, red);
    return cudaGetLastError();
}
cudaError_t launch_update_ur(const LevelT<double>& L, const Ctl* ctl, const double* p, const double* q, double* u,
                             double* r, const Red& red, cudaStream_t s)
{
    k_update_ur<<<RGRID(L)>>>(L, ctl, p, q, u, r, red);
    return cudaGetLastError();
}
cudaError_t launch_dot_rz(const LevelT<double>& L, const double* r, const double* z, const Red& red, cudaStream_t s)
{
    k_dot_rz<<<RGRID(L)>>>(L, r, z, red);
    return cudaGetLastError();
}
cudaError_t launch_update_p(const LevelT<double>& L, const Ctl* ctl, const double* z, double* p, cudaStream_t s)
{
    k_update_p<<<GRID(L)>>>(L, ctl, z, p);
    return cudaGetLastError();
}
// the row-per-warp form: grid and prefetch distance (half the rows the device holds resident;
// none on levels too small for the prefetched lines to stay inside the arrays)
static unsigned apply_rows_grid(const LevelT<float>& L)
{
    const size_t rows = (size_t)(L.ny - 2) * (L.nz - 2);
    return (unsigned)std::min((rows + 7) / 8, (L.N() + 255) / 256);
}

template <int LS, int V, typename K>
static cudaError_t apply_rows_pf(const LevelT<float>& L, K kernel, int* pf)
{
    static int pf_rows[64] = {0};
    *pf = 0;
    if (L.nx < 64 || L.ny < 8) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (pf_rows[dev] == 0) {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        pf_rows[dev] = std::max(1, per_sm * sms * 8 / 2);
    }
    *pf = pf_rows[dev];
    return cudaSuccess;
}

template <int LS, int V>
static cudaError_t launch_apply_dot32_rows(const LevelT<float>& L, const float* p, float* q, const Red& red, cudaStream_t s)
{
    int pf = 0;
    const cudaError_t e = apply_rows_pf<LS, V>(L, k_apply_dot32_rows<LS, V>, &pf);
    if (e != cudaSuccess) return e;
    k_apply_dot32_rows<LS, V><<<apply_rows_grid(L), 256, 0, s>>>(L, p, q, red, pf);
    return cudaGetLastError();
}

// the plane-staged form: geometry, dynamic shared memory and grid (one wave, at most one block
// per ceil(N / 256) nodes: the reduction's partials)
constexpr size_t AS_SMEM_MAX = 200 * 1024;

// geometry of one storage order on a level
template <int LS>
static void apply_stage_geom(const LevelT<float>& L, ApplyGeom& g, size_t& smem)
{
    const int nx = L.nx;
    g.tiles_j = (L.ny - 2 + AS_R - 1) / AS_R;
    const unsigned run = LS ? (unsigned)(((AS_R + 2) * nx + 1) / 2) : (unsigned)((AS_R + 2) * nx);
    g.slot = (run + 8u + 3u) & ~3u;
    g.hx1 = ((nx - 1) / 2 + 3) & ~3;
    smem = sizeof(float) * ((size_t)(LS ? 2 : 1) * AS_NS * g.slot + 8 * (size_t)g.hx1);
}

template <int V, int LS>
__global__ void __launch_bounds__(256) k_apply_stage(LevelT<float> L, const float* __restrict__ p, float* __restrict__ q,
                                                     Red red, ApplyGeom g, int* __restrict__ status);

// The grid: one wave of the blocks both storage orders hold resident (the fewer of the two), at
// most one block per ceil(N / 256) nodes (the reduction's partials).  The block-to-work map, and
// with it the order of the sums, thus depends on the grid shape alone -- never on the storage
// order or on a lockstep batch -- so every form of the solve forms the same dot products.
template <int V>
static cudaError_t apply_stage_plan(const LevelT<float>& L, int& chunk, unsigned& blocks)
{
    static int cache[64][3] = {{0, 0, 0}};   // nx, ny, blocks per SM
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int per_sm = 0;
    if (cache[dev][0] == L.nx && cache[dev][1] == L.ny) {
        per_sm = cache[dev][2];
    } else {
        ApplyGeom g0, g1;
        size_t m0 = 0, m1 = 0;
        apply_stage_geom<0>(L, g0, m0);
        apply_stage_geom<1>(L, g1, m1);
        if (m0 > AS_SMEM_MAX || m1 > AS_SMEM_MAX) return cudaErrorInvalidValue;
        int a0 = 0, a1 = 0;
        e = cudaFuncSetAttribute(k_apply_stage<V, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AS_SMEM_MAX);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_apply_stage<V, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AS_SMEM_MAX);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a0, k_apply_stage<V, 0>, 256, m0);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a1, k_apply_stage<V, 1>, 256, m1);
        if (e != cudaSuccess) return e;
        per_sm = std::max(1, std::min(a0, a1));
        cache[dev][0] = L.nx;
        cache[dev][1] = L.ny;
        cache[dev][2] = per_sm;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int tiles_j = (L.ny - 2 + AS_R - 1) / AS_R;
    const int planes = L.nz - 2;
    const size_t cap = std::min<size_t>((size_t)per_sm * sms, (L.N() + 255) / 256);
    const int chunks0 = (int)std::max<size_t>(1, std::min<size_t>(planes, cap / tiles_j));
    chunk = (planes + chunks0 - 1) / chunks0;
    blocks = (unsigned)(tiles_j * ((planes + chunk - 1) / chunk));
    return cudaSuccess;
}

static bool apply_stage_ok(const LevelT<float>& L, const float* p)
{
    return split_stage_ok(L.nx, L.ny, L.nz) && !((uintptr_t)p & 15u);
}

template <int V, int LS>
static cudaError_t launch_apply_stage(const LevelT<float>& L, const float* p, float* q, const Red& red, int* status,
                                      cudaStream_t s)
{
    ApplyGeom g;
    size_t smem = 0;
    unsigned blocks = 0;
    apply_stage_geom<LS>(L, g, smem);
    cudaError_t e = apply_stage_plan<V>(L, g.chunk, blocks);
    if (e != cudaSuccess) return e;
    k_apply_stage<V, LS><<<blocks, 256, smem, s>>>(L, p, q, red, g, status);
    return cudaGetLastError();
}

cudaError_t launch_apply_dot32(const LevelT<float>& L, const float* p, float* q, const Red& red, cudaStream_t s,
                               int* status)
{
    if (apply_stage_ok(L, p)) {
#define LASTO_APPLY_STAGE(VV)                                                                                       \
    case VV:                                                                                                        \
        return L.lsh ? launch_apply_stage<VV, 1>(L, p, q, red, status, s) : launch_apply_stage<VV, 0>(L, p, q, red, status, s);
        switch (split_rows_v(L.nx)) {
            LASTO_APPLY_STAGE(1)
            LASTO_APPLY_STAGE(2)
            LASTO_APPLY_STAGE(3)
            LASTO_APPLY_STAGE(4)
            LASTO_APPLY_STAGE(5)
            LASTO_APPLY_STAGE(6)
            LASTO_APPLY_STAGE(7)
            LASTO_APPLY_STAGE(8)
            default: break;
        }
#undef LASTO_APPLY_STAGE
    }
    if (L.ny >= 3 && L.nz >= 3) {
#define LASTO_APPLY_ROWS(VV)                                                                       \
    case VV:                                                                                       \
        return L.lsh ? launch_apply_dot32_rows<1, VV>(L, p, q, red, s) : launch_apply_dot32_rows<0, VV>(L, p, q, red, s);
        switch (split_rows_v(L.nx)) {
            LASTO_APPLY_ROWS(1)
            LASTO_APPLY_ROWS(2)
            LASTO_APPLY_ROWS(3)
            LASTO_APPLY_ROWS(4)
            LASTO_APPLY_ROWS(5)
            LASTO_APPLY_ROWS(6)
            LASTO_APPLY_ROWS(7)
            LASTO_APPLY_ROWS(8)
            default: break;
        }
#undef LASTO_APPLY_ROWS
    }
    // rows of more than 513 nodes
    if (L.lsh)
        k_apply_dot32<1><<<vec_grid(L.N()), NT, 0, s>>>(L, p, q, red);
    else
        k_apply_dot32<0><<<vec_grid(L.N()), NT, 0, s>>>(L, p, q, red);
    return cudaGetLastError();
}
cudaError_t launch_update_er32(const LevelT<float>& L, const Ctl* ctl, const float* p, const float* q, float* e,
                               float* r, const Red& red, cudaStream_t s)
{
    if (L.lsh)
        k_update_er32<1><<<vec_grid(L.N()), NT, 0, s>>>(L, ctl, p, q, e, r, red);
    else
        k_update_er32<0><<<vec_grid(L.N()), NT, 0, s>>>(L, ctl, p, q, e, r, red);
    return cudaGetLastError();
}
cudaError_t launch_dot32(const LevelT<float>& L, const float* r, const float* z, const Red& red, cudaStream_t s)
{
    if (L.lsh)
        k_dot32<1><<<vec_grid(L.N()), NT, 0, s>>>(L, r, z, red);
    else
        k_dot32<0><<<vec_grid(L.N()), NT, 0, s>>>(L, r, z, red);
    return cudaGetLastError();
}
cudaError_t launch_update_p32(const LevelT<float>& L, const Ctl* ctl, const float* z, float* p, cudaStream_t s)
{
    const unsigned g = (unsigned)((L.N() + NT * VU - 1) / (NT * VU));
    if (L.lsh)
        k_update_p32<1><<<g, NT, 0, s>>>(L, ctl, z, p);
    else
        k_update_p32<0><<<g, NT, 0, s>>>(L, ctl, z, p);
    return cudaGetLastError();
}
cudaError_t launch_add_correction(size_t N, double* u, float* e, unsigned h32, cudaStream_t s)
{
    k_add_correction<<<(unsigned)((N + NT - 1) / NT), NT, 0, s>>>(N, u, e, h32);
    return cudaGetLastError();
}
cudaError_t launch_to_f32(const double* a, float* b, size_t n, cudaStream_t s)
{
    k_to_f32<<<(unsigned)((n + NT - 1) / NT), NT, 0, s>>>(a, b, n);
    return cudaGetLastError();
}

__global__ void k_ctl_init(Ctl* ctl, double tol, double tol_iter, int max_iter)
{
    Ctl& c = *ctl;
    c.tol = tol;
    c.tol_iter = tol_iter;
    c.max_iter = max_iter;
    c.iter = 0;
    c.status = LASTO_ERR_NOT_CONVERGED;
    c.done = 0;
    c.rz = 1.0;
    c.alpha = c.beta = 0.0;
    c.rel = c.true_rel = -1.0;
    c.rz_in = 1.0;
    c.alpha_in = c.beta_in = c.rr0_in = 0.0;
    c.tol_in = 2e-5;
    c.iter_in = 0;
    c.max_in = 40;
    c.outer = 0;
    c.go_in = 0;
}

cudaError_t launch_ctl_init(Ctl* ctl, double tol, double tol_iter, int max_iter, cudaStream_t s)
{
    k_ctl_init<<<1, 1, 0, s>>>(ctl, tol, tol_iter, max_iter);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- lockstep batches
__device__ __forceinline__ bool bat_on(const Ctl* c, int mode)
{
    return mode == BAT_INNER ? c->go_in != 0 : c->done == 0;
}

__global__ void __launch_bounds__(512) k_rbgs_bat(const __grid_constant__ BatPack<BatLevel> pk, int colour, size_t nhalf)
{
    const BatLevel& a = pk.m[blockIdx.y];
    if (!bat_on(a.ctl, BAT_INNER)) return;
    k_rbgs_body<float, 0>(a.V, a.u, a.b, colour, nhalf);
}

template <int V>
__global__ void __launch_bounds__(256) k_rbgs_split_rows_bat(const __grid_constant__ BatPack<BatLevel> pk, int colour, int pf)
{
    const BatLevel& a = pk.m[blockIdx.y];
    if (!bat_on(a.ctl, BAT_INNER)) return;
    k_rbgs_split_rows_body<V>(a.V, a.u, a.b, colour, pf);
}

template <int LS, int RED_ONLY>
__global__ void __launch_bounds__(256) k_resid_restrict_rows_bat(const __grid_constant__ BatPack<BatLevel> pk)
{
    const BatLevel& a = pk.m[blockIdx.y];
    if (!bat_on(a.ctl, BAT_INNER)) return;
    k_resid_restrict_rows_body<LS, RED_ONLY>(a.V, a.VC, a.u, a.b, a.bc, a.uc);
}

template <int LS>
__global__ void __launch_bounds__(256) k_prolong_add_rows_bat(const __grid_constant__ BatPack<BatLevel> pk)
{
    const BatLevel& a = pk.m[blockIdx.y];
    if (!bat_on(a.ctl, BAT_INNER)) return;
    k_prolong_add_rows_body<LS>(a.V, a.VC, a.uc, a.u, 0);
}

__global__ void __launch_bounds__(BOT_NT) k_bottom_bat(const BatBottom* __restrict__ m)
{
    const BatBottom& a = m[blockIdx.x];
    if (!bat_on(a.ctl, BAT_INNER)) return;
    k_bottom_body<float>(a.a);
}

__global__ void __launch_bounds__(NT) k_zero_bat(const __grid_constant__ BatPack<BatVec> pk, size_t n, int which, int mode)
{
    const BatVec& a = pk.m[blockIdx.y];
    if (!bat_on(a.ctl, mode)) return;
    float* x = which == 0 ? a.u32 : a.p32;
    GRID_STRIDE(P, n) x[P] = 0.0f;
}

template <int LS>
__global__ void __launch_bounds__(NT, VEC_MIN_BLOCKS) k_dot32_bat(const __grid_constant__ BatPack<BatVec> pk, int with_z, int op, int mode)
{
    const BatVec& a = pk.m[blockIdx.y];
    if (!bat_on(a.ctl, mode)) return;
    const Red red{a.part, a.counter, a.ctl, op, 0, 0};
    k_dot32_body<LS>(a.V32, a.b32, with_z ? a.u32 : nullptr, red);
}

template <int LS>
__global__ void __launch_bounds__(NT) k_update_p32_bat(const __grid_constant__ BatPack<BatVec> pk)
{
    const BatVec& a = pk.m[blockIdx.y];
    if (!bat_on(a.ctl, BAT_INNER)) return;
    k_update_p32_body<LS>(a.V32, a.ctl, a.u32, a.p32);
}

template <int LS>
__global__ void __launch_bounds__(NT, VEC_MIN_BLOCKS) k_apply_dot32_bat(const __grid_constant__ BatPack<BatVec> pk)
{
    const BatVec& a = pk.m[blockIdx.y];
    if (!bat_on(a.ctl, BAT_INNER)) return;
    const Red red{a.part, a.counter, a.ctl, FIN_IN_ALPHA, 0, 0};
    k_apply_dot32_body<LS>(a.V32, a.p32, a.q32, red);
}

template <int V, int LS>
__global__ void __launch_bounds__(256) k_apply_stage_bat(const __grid_constant__ BatPack<BatVec> pk, ApplyGeom g)
{
    const BatVec& a = pk.m[blockIdx.y];
    if (!bat_on(a.ctl, BAT_INNER)) return;
    const Red red{a.part, a.counter, a.ctl, FIN_IN_ALPHA, 0, 0};
    k_apply_stage_body<V, LS>(a.V32, a.p32, a.q32, red, g, a.status);
}

template <int LS, int V>
__global__ void __launch_bounds__(256) k_apply_dot32_rows_bat(const __grid_constant__ BatPack<BatVec> pk, int pf)
{
    const BatVec& a = pk.m[blockIdx.y];
    if (!bat_on(a.ctl, BAT_INNER)) return;
    const Red red{a.part, a.counter, a.ctl, FIN_IN_ALPHA, 0, 0};
    k_apply_dot32_rows_body<LS, V>(a.V32, a.p32, a.q32, red, pf);
}

template <int LS>
__global__ void __launch_bounds__(NT, VEC_MIN_BLOCKS) k_update_er32_bat(const __grid_constant__ BatPack<BatVec> pk)
{
    const BatVec& a = pk.m[blockIdx.y];
    if (!bat_on(a.ctl, BAT_INNER)) return;
    const Red red{a.part, a.counter, a.ctl, FIN_IN_CHECK, 0, 0};
    k_update_er32_body<LS>(a.V32, a.ctl, a.p32, a.q32, a.e32, a.b32, red);
}

__global__ void __launch_bounds__(NT) k_add_correction_bat(const __grid_constant__ BatPack<BatVec> pk, size_t n, unsigned h32)
{
    const BatVec& a = pk.m[blockIdx.y];
    if (!bat_on(a.ctl, BAT_OUTER)) return;
    k_add_correction_body(n, a.u, a.e32, h32);
}

__global__ void __launch_bounds__(NT) k_resid_norm_bat(const __grid_constant__ BatPack<BatVec> pk, unsigned h32)
{
    const BatVec& a = pk.m[blockIdx.y];
    if (!bat_on(a.ctl, BAT_OUTER)) return;
    const Red red{a.part, a.counter, a.ctl, FIN_OUTER, 0, 0};
    k_resid_norm_body(a.V64, a.u, a.b, a.r, a.b32, h32, red);
}

__global__ void k_any_bat(Ctl* const* __restrict__ ctls, int nm, int mode, cudaGraphConditionalHandle cond)
{
    int any = 0;
    for (int c = 0; c < nm; c++) any |= bat_on(ctls[c], mode) ? 1 : 0;
    cudaGraphSetConditional(cond, (unsigned)any);
}

cudaError_t launch_rbgs_bat(const LevelT<float>& V0, const BatPack<BatLevel>& m, int nm, int colour, int nt, cudaStream_t s)
{
    if (nm < 1 || nm > BAT_MAX) return cudaErrorInvalidValue;
    if (V0.lsh) {
        int pf = 0;
        cudaError_t e = cudaSuccess;
        const unsigned g = (unsigned)(((size_t)(V0.ny - 2) * (V0.nz - 2) + 7) / 8);
#define LASTO_SPLIT_BAT(VV)                                                              \
    case VV:                                                                             \
        e = split_rows_pf<VV>(&pf);                                                      \
        if (e != cudaSuccess) return e;                                                  \
        k_rbgs_split_rows_bat<VV><<<dim3(g, (unsigned)nm), 256, 0, s>>>(m, colour, pf);   \
        break;
        switch (split_rows_v(V0.nx)) {
            LASTO_SPLIT_BAT(1)
            LASTO_SPLIT_BAT(2)
            LASTO_SPLIT_BAT(3)
            LASTO_SPLIT_BAT(4)
            LASTO_SPLIT_BAT(5)
            LASTO_SPLIT_BAT(6)
            LASTO_SPLIT_BAT(7)
            LASTO_SPLIT_BAT(8)
            default: return cudaErrorInvalidValue;
        }
#undef LASTO_SPLIT_BAT
        return cudaGetLastError();
    }
    if (nt < 32 || nt > 512 || nt % 32) nt = 256;
    const size_t nhalf = (V0.N() + 1 - colour) / 2;
    k_rbgs_bat<<<dim3((unsigned)((nhalf + nt - 1) / nt), (unsigned)nm), nt, 0, s>>>(m, colour, nhalf);
    return cudaGetLastError();
}

cudaError_t launch_resid_restrict_bat(const LevelT<float>& F0, const LevelT<float>& C0, const BatPack<BatLevel>& m, int nm,
                                      bool red_only, cudaStream_t s)
{
    if (nm < 1 || nm > BAT_MAX || C0.lsh) return cudaErrorInvalidValue;
    const dim3 g((unsigned)(((size_t)C0.ny * C0.nz + 7) / 8), (unsigned)nm);
    if (F0.lsh && red_only)
        k_resid_restrict_rows_bat<1, 1><<<g, 256, 0, s>>>(m);
    else if (F0.lsh)
        k_resid_restrict_rows_bat<1, 0><<<g, 256, 0, s>>>(m);
    else if (red_only)
        k_resid_restrict_rows_bat<0, 1><<<g, 256, 0, s>>>(m);
    else
        k_resid_restrict_rows_bat<0, 0><<<g, 256, 0, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_prolong_add_bat(const LevelT<float>& F0, const LevelT<float>& C0, const BatPack<BatLevel>& m, int nm,
                                   cudaStream_t s)
{
    if (nm < 1 || nm > BAT_MAX || C0.lsh || F0.ny < 3 || F0.nz < 3) return cudaErrorInvalidValue;
    const dim3 g((unsigned)(((size_t)(F0.ny - 2) * (F0.nz - 2) + 7) / 8), (unsigned)nm);
    if (F0.lsh)
        k_prolong_add_rows_bat<1><<<g, 256, 0, s>>>(m);
    else
        k_prolong_add_rows_bat<0><<<g, 256, 0, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_bottom_bat(const BottomArgs<float>& a0, const BatBottom* m, int nm, cudaStream_t s)
{
    const size_t smem = bottom_smem_bytes(a0);
    if (smem > 200 * 1024 || nm < 1) return cudaErrorInvalidValue;
    for (int q = 0; q < a0.nlev; q++)
        if (a0.lv[q].lsh) return cudaErrorInvalidValue;
    k_bottom_bat<<<(unsigned)nm, BOT_NT, smem, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_zero_bat(const BatPack<BatVec>& m, int nm, size_t n, int which, int mode, cudaStream_t s)
{
    if (nm < 1 || nm > BAT_MAX) return cudaErrorInvalidValue;
    k_zero_bat<<<dim3(red_grid(n), (unsigned)nm), NT, 0, s>>>(m, n, which, mode);
    return cudaGetLastError();
}

cudaError_t launch_dot32_bat(const LevelT<float>& V0, const BatPack<BatVec>& m, int nm, int with_z, int op, int mode,
                             cudaStream_t s)
{
    const dim3 g(vec_grid(V0.N()), (unsigned)nm);
    if (V0.lsh)
        k_dot32_bat<1><<<g, NT, 0, s>>>(m, with_z, op, mode);
    else
        k_dot32_bat<0><<<g, NT, 0, s>>>(m, with_z, op, mode);
    return cudaGetLastError();
}

cudaError_t launch_update_p32_bat(const LevelT<float>& V0, const BatPack<BatVec>& m, int nm, cudaStream_t s)
{
    const dim3 g((unsigned)((V0.N() + NT * VU - 1) / (NT * VU)), (unsigned)nm);
    if (V0.lsh)
        k_update_p32_bat<1><<<g, NT, 0, s>>>(m);
    else
        k_update_p32_bat<0><<<g, NT, 0, s>>>(m);
    return cudaGetLastError();
}

template <int LS, int V>
static cudaError_t launch_apply_dot32_rows_bat(const LevelT<float>& V0, const BatPack<BatVec>& m, int nm, cudaStream_t s)
{
    int pf = 0;
    const cudaError_t e = apply_rows_pf<LS, V>(V0, k_apply_dot32_rows<LS, V>, &pf);
    if (e != cudaSuccess) return e;
    k_apply_dot32_rows_bat<LS, V><<<dim3(apply_rows_grid(V0), (unsigned)nm), 256, 0, s>>>(m, pf);
    return cudaGetLastError();
}

template <int V, int LS>
static cudaError_t launch_apply_stage_bat(const LevelT<float>& V0, const BatPack<BatVec>& m, int nm, cudaStream_t s)
{
    static bool attr[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        e = cudaFuncSetAttribute(k_apply_stage_bat<V, LS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AS_SMEM_MAX);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    ApplyGeom g;
    size_t smem = 0;
    unsigned blocks = 0;
    apply_stage_geom<LS>(V0, g, smem);
    e = apply_stage_plan<V>(V0, g.chunk, blocks);   // the members' own grid
    if (e != cudaSuccess) return e;
    k_apply_stage_bat<V, LS><<<dim3(blocks, (unsigned)nm), 256, smem, s>>>(m, g);
    return cudaGetLastError();
}

cudaError_t launch_apply_dot32_bat(const LevelT<float>& V0, const BatPack<BatVec>& m, int nm, cudaStream_t s)
{
    if (nm < 1 || nm > BAT_MAX) return cudaErrorInvalidValue;
    bool aligned = true;
    for (int q = 0; q < nm; q++) aligned = aligned && apply_stage_ok(m.m[q].V32, m.m[q].p32);
    if (aligned) {
#define LASTO_APPLY_STAGE(VV)                                                                                  \
    case VV:                                                                                                   \
        return V0.lsh ? launch_apply_stage_bat<VV, 1>(V0, m, nm, s) : launch_apply_stage_bat<VV, 0>(V0, m, nm, s);
        switch (split_rows_v(V0.nx)) {
            LASTO_APPLY_STAGE(1)
            LASTO_APPLY_STAGE(2)
            LASTO_APPLY_STAGE(3)
            LASTO_APPLY_STAGE(4)
            LASTO_APPLY_STAGE(5)
            LASTO_APPLY_STAGE(6)
            LASTO_APPLY_STAGE(7)
            LASTO_APPLY_STAGE(8)
            default: break;
        }
#undef LASTO_APPLY_STAGE
    }
    if (V0.ny >= 3 && V0.nz >= 3) {
#define LASTO_APPLY_ROWS(VV)                                                                          \
    case VV:                                                                                          \
        return V0.lsh ? launch_apply_dot32_rows_bat<1, VV>(V0, m, nm, s) : launch_apply_dot32_rows_bat<0, VV>(V0, m, nm, s);
        switch (split_rows_v(V0.nx)) {
            LASTO_APPLY_ROWS(1)
            LASTO_APPLY_ROWS(2)
            LASTO_APPLY_ROWS(3)
            LASTO_APPLY_ROWS(4)
            LASTO_APPLY_ROWS(5)
            LASTO_APPLY_ROWS(6)
            LASTO_APPLY_ROWS(7)
            LASTO_APPLY_ROWS(8)
            default: break;
        }
#undef LASTO_APPLY_ROWS
    }
    const dim3 g(vec_grid(V0.N()), (unsigned)nm);
    if (V0.lsh)
        k_apply_dot32_bat<1><<<g, NT, 0, s>>>(m);
    else
        k_apply_dot32_bat<0><<<g, NT, 0, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_update_er32_bat(const LevelT<float>& V0, const BatPack<BatVec>& m, int nm, cudaStream_t s)
{
    const dim3 g(vec_grid(V0.N()), (unsigned)nm);
    if (V0.lsh)
        k_update_er32_bat<1><<<g, NT, 0, s>>>(m);
    else
        k_update_er32_bat<0><<<g, NT, 0, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_outer_bat(const LevelT<double>& V0, const BatPack<BatVec>& m, int nm, unsigned h32, cudaStream_t s)
{
    const size_t N = V0.N();
    k_add_correction_bat<<<dim3((unsigned)((N + NT - 1) / NT), (unsigned)nm), NT, 0, s>>>(m, N, h32);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_resid_norm_bat<<<dim3(resid_rows_grid(V0), (unsigned)nm), NT, 0, s>>>(m, h32);
    return cudaGetLastError();
}

cudaError_t launch_any_bat(Ctl* const* ctls, int nm, int mode, cudaGraphConditionalHandle cond, cudaStream_t s)
{
    k_any_bat<<<1, 1, 0, s>>>(ctls, nm, mode, cond);
    return cudaGetLastError();
}

void init_bat_attributes()
{
    cudaFuncSetAttribute(k_bottom_bat, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

// ---------------------------------------------------------------- instantiations
#define INST(T)                                                                                              \
    template cudaError_t launch_resid_restrict<T>(const LevelT<T>&, const LevelT<T>&, const T*, const T*, T*, T*, \
                                                  bool, cudaStream_t, T*, int*);                            \
    template cudaError_t launch_bottom<T>(const BottomArgs<T>&, cudaStream_t);                              \
    template cudaError_t launch_rbgs<T>(const LevelT<T>&, T*, const T*, int, cudaStream_t, int, int*);               \
    template cudaError_t launch_residual<T>(const LevelT<T>&, const T*, const T*, T*, cudaStream_t);        \
    template cudaError_t launch_apply<T>(const LevelT<T>&, const T*, T*, cudaStream_t);                     \
    template cudaError_t launch_restrict<T>(const LevelT<T>&, const LevelT<T>&, const T*, T*, cudaStream_t); \
    template cudaError_t launch_prolong_add<T>(const LevelT<T>&, const LevelT<T>&, const T*, T*, cudaStream_t, int*); \
    template cudaError_t launch_coarse_apply<T>(const LevelT<T>&, const CoarseEig*, const T*, T*, bool, cudaStream_t);
INST(double)
INST(float)

}  // namespace lasto
