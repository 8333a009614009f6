// Fused red-black Gauss-Seidel smoother on z-slabs staged in shared memory
// (Section 3: the finite-difference multigrid smoother).
//
// One pass applies NS full sweeps (2 NS colour stages) and reads u_in and b once and
// writes u_out once, instead of 2 NS in-place half-sweep launches that each stream the
// whole grid.  A CTA owns an (x, y) tile and a range of z planes.  It walks z upwards,
// keeping a rolling window of planes in shared memory: plane p arrives by cp.async while
// the stages run on the planes below it.  Stage s (colour (first + s) mod 2) runs one
// plane behind stage s - 1, and on the tile widened by 2 NS - 1 - s nodes in x and y (and
// as many planes past the z range), so that every value the last stage needs is computed
// inside the CTA from u_in alone.  These halo nodes are computed by the neighbouring CTA
// too, with the same operands and the same arithmetic, so the result does not depend on
// the tiling: it is bitwise the in-place sweep (each update reads the other colour's newest
// values, as Gauss-Seidel does).  u_in and u_out must be different arrays; every node of
// u_out is written (faces copied from u_in).
#include <algorithm>

#include "internal.cuh"

namespace lasto {

namespace {

constexpr int SLAB_NT = 256;

__device__ __forceinline__ void cp_async(float* dst, const float* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async(double* dst, const double* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <typename T, int NS>
__global__ void __launch_bounds__(SLAB_NT) k_rb_slab(LevelT<T> L, const T* __restrict__ uin, T* __restrict__ uout,
                                                     const T* __restrict__ b, int first, int zero_in, int tx, int ty,
                                                     int kz)
{
    extern __shared__ __align__(16) unsigned char slab_smem[];
    T* win = reinterpret_cast<T*>(slab_smem);
    constexpr int H = 2 * NS;        // halo rings loaded around the tile
    constexpr int W = 2 * NS + 3;    // planes in the rolling window
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int RX = tx + 2 * H, RY = ty + 2 * H, RP = RX * RY;
    const int i0 = blockIdx.x * tx, j0 = blockIdx.y * ty, k0 = blockIdx.z * kz;
    const int ti1 = min(i0 + tx, nx), tj1 = min(j0 + ty, ny), k1 = min(k0 + kz, nz);
    const int gx = i0 - H, gy = j0 - H;   // global (i, j) of window cell (0, 0)
    const size_t sy = (size_t)nx, sz = (size_t)nx * ny;
    const int tid = threadIdx.x;

    auto slot = [&](int q) { return win + (size_t)(((q % W) + W) % W) * RP; };

    // issue the loads of plane q into its window slot (cells outside the grid stay unset:
    // only interior nodes are updated and their neighbours lie inside the grid)
    auto load = [&](int q) {
        if (q < 0 || q >= nz) return;
        T* dst = slot(q);
        const int xa = max(gx, 0) - gx, xb = min(gx + RX, nx) - gx;
        const int ya = max(gy, 0) - gy, yb = min(gy + RY, ny) - gy;
        const int w = xb - xa, cnt = w * (yb - ya);
        for (int e = tid; e < cnt; e += SLAB_NT) {
            const int y = ya + e / w, x = xa + e % w;
            if (zero_in) {
                dst[y * RX + x] = T(0);
            } else {
                cp_async(dst + y * RX + x, uin + (size_t)q * sz + (size_t)(gy + y) * sy + (gx + x));
            }
        }
    };

    const int pstart = k0 - H, pend = k1 - 1 + H;
    load(pstart);
    cp_async_commit();
    for (int p = pstart; p <= pend; p++) {
        load(p + 1);
        cp_async_commit();
        cp_async_wait_prev();
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 2 * NS; s++) {
            const int q = p - 1 - s;
            const int R = 2 * NS - 1 - s;
            if (q < max(1, k0 - R) || q > min(nz - 2, k1 - 1 + R)) continue;   // uniform over the block
            const int c = (first + s) & 1;
            const int ia = max(1, i0 - R), ib = min(nx - 2, ti1 - 1 + R);
            const int ja = max(1, j0 - R), jb = min(ny - 2, tj1 - 1 + R);
            if (ia <= ib && ja <= jb) {
                const int mc = (ib - ia) / 2 + 1, rows = jb - ja + 1;
                T* pc = slot(q);
                const T* pm = slot(q - 1);
                const T* pp = slot(q + 1);
                const T cmz = L.ax[2].cm[q], cpz = L.ax[2].cp[q];
                for (int e = tid; e < rows * mc; e += SLAB_NT) {
                    const int jr = e / mc, j = ja + jr;
                    const int i = ia + ((c - ia - j - q) & 1) + 2 * (e - jr * mc);
                    if (i > ib) continue;
                    const int o = (j - gy) * RX + (i - gx);
                    // the six neighbour terms in the fixed order x-, x+, y-, y+, z-, z+
                    T t = L.ax[0].cm[i] * pc[o - 1];
                    t = fma(L.ax[0].cp[i], pc[o + 1], t);
                    t = fma(L.ax[1].cm[j], pc[o - RX], t);
                    t = fma(L.ax[1].cp[j], pc[o + RX], t);
                    t = fma(cmz, pm[o], t);
                    t = fma(cpz, pp[o], t);
                    const size_t P = (size_t)q * sz + (size_t)j * sy + i;
                    const T acc = b[P] - t;
                    if constexpr (sizeof(T) == 8) {
                        pc[o] = acc * L.inv_diag[P];
                    } else {
                        pc[o] = rb_point32(acc, L.ax[0].dg[i] + L.ax[1].dg[j] + L.ax[2].dg[q]);
                    }
                }
            }
            __syncthreads();
        }
        // plane p - 2 NS has had its last stage: store the tile (faces unchanged)
        const int q = p - H;
        if (q >= k0 && q < k1) {
            const T* src = slot(q);
            const int w = ti1 - i0, cnt = w * (tj1 - j0);
            for (int e = tid; e < cnt; e += SLAB_NT) {
                const int y = e / w, x = e - y * w;
                uout[(size_t)q * sz + (size_t)(j0 + y) * sy + (i0 + x)] = src[(y + H) * RX + (x + H)];
            }
        }
        __syncthreads();
    }
}

// One full sweep per pass with the z column in registers.  A warp is one row of the
// block: lane px owns the node pair (i0 - 1 + 2 px, i0 + 2 px) of row j0 - 1 + py, one red
// and one black node in every plane; 32 lanes cover the 62-node tile plus one node each
// side, and the block's RY rows the tile's ty = RY - 2 rows plus one each side.  At step p
// a lane updates its red node of plane p-1 (x/y neighbours from shared plane A: the old
// values, plus one node of halo that the edge lanes bring), its black node of plane p-2
// (x/y neighbours from shared plane B: the red values published a step earlier), and
// writes plane p-2.  The pair's u and b (and the FP64 inverse diagonal) for planes
// p-3 .. p+2 form a register ring; the loop is unrolled over the ring length, so ring
// slots, shared slots and the colour of each node of the pair are constants of the
// unrolled step (the colour pattern also depends on RB = parity(i0 - 1 + j + k0) xor
// first, a template parameter).  Loads of plane p+2 are in flight for two steps; the halo
// arrives by cp.async.  One barrier per step orders every shared read after its write.
constexpr int COL_PX = 32;       // lanes per row (one warp)
constexpr int COL_TX = 2 * (COL_PX - 1);
constexpr int CR = 6;            // register ring and shared A ring: planes p-3 .. p+2

template <typename T, int RB>
__device__ __forceinline__ void col_sweep(const LevelT<T>& L, const T* __restrict__ uin, T* __restrict__ uout,
                                          const T* __restrict__ b, int zero_in, int k0, int k1, T* SA, T* SB,
                                          const T* ZC)
{
    const int RY = blockDim.y;
    const int TY = RY - 2;
    constexpr int AX = COL_TX + 4, BX = COL_TX + 2;
    const int AY = TY + 4, AP = AX * AY, BP = RY * BX;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int px = threadIdx.x, py = threadIdx.y;
    const int i0 = blockIdx.x * COL_TX, j0 = blockIdx.y * TY;
    const int ia = i0 - 1 + 2 * px, j = j0 - 1 + py;
    const size_t sy = (size_t)nx, sz = (size_t)nx * ny;
    const bool row_in = j >= 0 && j < ny;
    const bool in_a = row_in && ia >= 0 && ia < nx, in_b = row_in && ia + 1 < nx;
    const bool row_int = j >= 1 && j <= ny - 2;
    const bool int_a = row_int && ia >= 1 && ia <= nx - 2, int_b = row_int && ia + 1 >= 1 && ia + 1 <= nx - 2;
    const bool row_tile = py >= 1 && py <= TY;
    const bool wa = row_tile && px >= 1 && in_a, wb = row_tile && px <= COL_PX - 2 && in_b;
    const bool ua_ok = in_a && !zero_in, ub_ok = in_b && !zero_in;
    const int oA = (py + 1) * AX + 2 * px + 1, oB = py * BX + 2 * px;
    // per-thread offset of node a within a plane (ia may be -1: node b = rowoff + 1 is then
    // column 0; node a itself is never accessed when it lies outside the grid)
    const long long rowoff = (long long)min(max(j, 0), ny - 1) * nx + ia;
    const int ca = min(max(ia, 0), nx - 1), cb = min(max(ia + 1, 0), nx - 1), cj = min(max(j, 0), ny - 1);
    const T cmxa = L.ax[0].cm[ca], cpxa = L.ax[0].cp[ca], cmxb = L.ax[0].cm[cb], cpxb = L.ax[0].cp[cb];
    const T dga = L.ax[0].dg[ca], dgb = L.ax[0].dg[cb];
    const T cmy = L.ax[1].cm[cj], cpy = L.ax[1].cp[cj], dgy = L.ax[1].dg[cj];
    // halo roles
    const bool hl = px == 0 && row_in && i0 - 2 >= 0, hr = px == COL_PX - 1 && row_in && i0 + COL_TX + 1 < nx;
    const bool hd = py == 0 && j0 - 2 >= 0, hu = py == RY - 1 && j0 + TY + 1 < ny;
    const bool hd_a = hd && ia >= 0 && ia < nx, hd_b = hd && ia + 1 < nx;
    const bool hu_a = hu && ia >= 0 && ia < nx, hu_b = hu && ia + 1 < nx;
    const size_t hoff_l = (size_t)min(max(j, 0), ny - 1) * sy + (size_t)max(i0 - 2, 0);
    const size_t hoff_r = (size_t)min(max(j, 0), ny - 1) * sy + (size_t)min(i0 + COL_TX + 1, nx - 1);
    const long long hoff_d = (long long)max(j0 - 2, 0) * nx + ia;
    const long long hoff_u = (long long)min(j0 + TY + 1, ny - 1) * nx + ia;

    auto halo = [&](T* A, int q) {
        if (q < 0 || q >= nz) return;
        const long long off = (long long)q * (long long)sz;
        auto put = [&](bool ok, int o, long long g) {
            if (!ok) return;
            if (zero_in)
                A[o] = T(0);
            else
                cp_async(A + o, uin + off + g);
        };
        put(hl, (py + 1) * AX, (long long)hoff_l);
        put(hr, (py + 1) * AX + AX - 1, (long long)hoff_r);
        put(hd_a, 2 * px + 1, hoff_d);
        put(hd_b, 2 * px + 2, hoff_d + 1);
        put(hu_a, (AY - 1) * AX + 2 * px + 1, hoff_u);
        put(hu_b, (AY - 1) * AX + 2 * px + 2, hoff_u + 1);
    };

    T ua[CR], ub[CR], ba[CR], bb[CR], va[CR], vb[CR];
#pragma unroll
    for (int r = 0; r < CR; r++) ua[r] = ub[r] = ba[r] = bb[r] = va[r] = vb[r] = T(0);
    auto load = [&](int r, int q) {
        const bool qu = q >= 0 && q < nz, qb = q >= 1 && q <= nz - 2;
        const long long off = (long long)q * (long long)sz + rowoff;
        ua[r] = (ua_ok && qu) ? uin[off] : T(0);
        ub[r] = (ub_ok && qu) ? uin[off + 1] : T(0);
        ba[r] = (int_a && qb) ? b[off] : T(0);
        bb[r] = (int_b && qb) ? b[off + 1] : T(0);
        if constexpr (sizeof(T) == 8) {
            va[r] = (int_a && qb) ? L.inv_diag[off] : T(0);
            vb[r] = (int_b && qb) ? L.inv_diag[off + 1] : T(0);
        }
    };
    // prologue: ring slot r <-> plane k0-3+r at step p = k0; A slot of plane q = (q-k0+3) mod CR
#pragma unroll
    for (int r = 0; r < CR - 1; r++) load(r, k0 - 3 + r);
    for (int q = k0 - 1; q <= k0 + 1; q++) {
        halo(SA + (q - k0 + 3) * AP, q);
        cp_async_commit();
    }

    for (int p0 = k0; p0 <= k1 + 1; p0 += CR) {
#pragma unroll
        for (int s = 0; s < CR; s++) {
            const int p = p0 + s;
            if (p > k1 + 1) break;
            const int r3 = s % CR, r2 = (s + 1) % CR, r1 = (s + 2) % CR, r0 = (s + 3) % CR, rn = (s + 5) % CR;
            load(rn, p + 2);
            halo(SA + ((s + 5) % CR) * AP, p + 2);
            cp_async_commit();
            T* A = SA + ((s + 2) % CR) * AP;    // plane p-1
            A[oA] = ua[r1];
            A[oA + 1] = ub[r1];
            asm volatile("cp.async.wait_group 3;\n" ::: "memory");
            __syncthreads();
            const T* Bp = SB + ((s + 1) & 1) * BP;
            T* Bn = SB + (s & 1) * BP;
            // red node of plane p-1: node a when RB + s + 1 is even
            const bool red_a = ((RB + s + 1) & 1) == 0;
            const int q = p - 1;
            if (q >= max(1, k0 - 1) && q <= min(nz - 2, k1) && (red_a ? int_a : int_b)) {
                const T* zc = ZC + 3 * (q - k0 + 2);
                T t;
                if (red_a) {
                    t = cmxa * A[oA - 1];
                    t = fma(cpxa, ub[r1], t);
                    t = fma(cmy, A[oA - AX], t);
                    t = fma(cpy, A[oA + AX], t);
                    t = fma(zc[0], ua[r2], t);
                    t = fma(zc[1], ua[r0], t);
                    const T acc = ba[r1] - t;
                    if constexpr (sizeof(T) == 8)
                        ua[r1] = acc * va[r1];
                    else
                        ua[r1] = rb_point32(acc, dga + dgy + zc[2]);
                } else {
                    t = cmxb * ua[r1];
                    t = fma(cpxb, A[oA + 2], t);
                    t = fma(cmy, A[oA + 1 - AX], t);
                    t = fma(cpy, A[oA + 1 + AX], t);
                    t = fma(zc[0], ub[r2], t);
                    t = fma(zc[1], ub[r0], t);
                    const T acc = bb[r1] - t;
                    if constexpr (sizeof(T) == 8)
                        ub[r1] = acc * vb[r1];
                    else
                        ub[r1] = rb_point32(acc, dgb + dgy + zc[2]);
                }
            }
            // black node of plane p-2 (tile nodes only): node a when RB + s is odd
            const bool blk_a = ((RB + s) & 1) == 1;
            const int q2 = p - 2;
            if (q2 >= max(1, k0) && q2 <= min(nz - 2, k1 - 1) && (blk_a ? (int_a && wa) : (int_b && wb))) {
                const T* zc = ZC + 3 * (q2 - k0 + 2);
                T t;
                if (blk_a) {
                    t = cmxa * Bp[oB - 1];
                    t = fma(cpxa, ub[r2], t);
                    t = fma(cmy, Bp[oB - BX], t);
                    t = fma(cpy, Bp[oB + BX], t);
                    t = fma(zc[0], ua[r3], t);
                    t = fma(zc[1], ua[r1], t);
                    const T acc = ba[r2] - t;
                    if constexpr (sizeof(T) == 8)
                        ua[r2] = acc * va[r2];
                    else
                        ua[r2] = rb_point32(acc, dga + dgy + zc[2]);
                } else {
                    t = cmxb * ua[r2];
                    t = fma(cpxb, Bp[oB + 2], t);
                    t = fma(cmy, Bp[oB + 1 - BX], t);
                    t = fma(cpy, Bp[oB + 1 + BX], t);
                    t = fma(zc[0], ub[r3], t);
                    t = fma(zc[1], ub[r1], t);
                    const T acc = bb[r2] - t;
                    if constexpr (sizeof(T) == 8)
                        ub[r2] = acc * vb[r2];
                    else
                        ub[r2] = rb_point32(acc, dgb + dgy + zc[2]);
                }
            }
            if (q2 >= k0 && q2 < k1) {
                const long long off = (long long)q2 * (long long)sz + rowoff;
                if (wa) uout[off] = ua[r2];
                if (wb) uout[off + 1] = ub[r2];
            }
            Bn[oB] = ua[r1];
            Bn[oB + 1] = ub[r1];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512)
    k_rb_col(LevelT<T> L, const T* __restrict__ uin, T* __restrict__ uout, const T* __restrict__ b, int first,
             int zero_in, int kz)
{
    extern __shared__ __align__(16) unsigned char col_smem[];
    const int RY = blockDim.y, TY = RY - 2;
    constexpr int AX = COL_TX + 4, BX = COL_TX + 2;
    const int AY = TY + 4;
    T* SA = reinterpret_cast<T*>(col_smem);   // [CR][AY][AX]
    T* SB = SA + CR * AX * AY;                 // [2][RY][BX]
    T* ZC = SB + 2 * RY * BX;                  // [kz + 4][3]: cm, cp, dg of planes k0-2 ..
    const int nz = L.nz;
    const int k0 = blockIdx.z * kz, k1 = min(k0 + kz, nz);
    const int tid = threadIdx.y * COL_PX + threadIdx.x;
    for (int e = tid; e < kz + 4; e += COL_PX * RY) {
        const int qc = min(max(k0 - 2 + e, 0), nz - 1);
        ZC[3 * e] = L.ax[2].cm[qc];
        ZC[3 * e + 1] = L.ax[2].cp[qc];
        ZC[3 * e + 2] = L.ax[2].dg[qc];
    }
    // colour pattern of the warp's pairs (uniform over the warp: one row, one parity of i)
    const int j = blockIdx.y * TY - 1 + (int)threadIdx.y;
    const int rb = ((blockIdx.x * COL_TX - 1 + j + k0) & 1) ^ (first & 1);
    if (rb)
        col_sweep<T, 1>(L, uin, uout, b, zero_in, k0, k1, SA, SB, ZC);
    else
        col_sweep<T, 0>(L, uin, uout, b, zero_in, k0, k1, SA, SB, ZC);
}

template <typename T, int NS>
void* slab_kernel()
{
    return reinterpret_cast<void*>(&k_rb_slab<T, NS>);
}

template <typename T>
void* col_kernel()
{
    return reinterpret_cast<void*>(&k_rb_col<T>);
}

}  // namespace

// ns = 1 runs the column kernel (tx = 62; block 32 x (ty + 2) threads); ns = 2 the z-slab
// window kernel (256 threads).
size_t slab_smem_bytes(const SlabShape& sh, size_t elem)
{
    if (sh.ns == 1) {
        const size_t AX = COL_TX + 4, AY = sh.ty + 4, BX = COL_TX + 2, RY = sh.ty + 2;
        return (CR * AX * AY + 2 * RY * BX + 3 * ((size_t)sh.kz + 4)) * elem;
    }
    const size_t H = 2 * (size_t)sh.ns;
    return (2 * (size_t)sh.ns + 3) * ((size_t)sh.tx + 2 * H) * ((size_t)sh.ty + 2 * H) * elem;
}

bool slab_shape_ok(const SlabShape& sh, size_t elem)
{
    if (sh.ns == 1)
        return sh.tx == COL_TX && sh.ty >= 1 && sh.kz >= 1 && sh.kz <= 4096 && COL_PX * (sh.ty + 2) <= (elem == 8 ? 256 : 512) &&
               slab_smem_bytes(sh, elem) <= SLAB_MAX_SMEM;
    return sh.ns == 2 && sh.tx >= 2 && sh.ty >= 1 && sh.kz >= 1 && sh.tx <= 512 && sh.ty <= 512 &&
           slab_smem_bytes(sh, elem) <= SLAB_MAX_SMEM;
}

SlabShape slab_default_shape(int ns, size_t elem)
{
    if (ns == 1) return SlabShape{COL_TX, elem == 8 ? 6 : 14, 32, 1};
    return SlabShape{64, 16, 32, 2};
}

void init_slab_attributes()
{
    cudaFuncSetAttribute(col_kernel<float>(), cudaFuncAttributeMaxDynamicSharedMemorySize, SLAB_MAX_SMEM);
    cudaFuncSetAttribute(col_kernel<double>(), cudaFuncAttributeMaxDynamicSharedMemorySize, SLAB_MAX_SMEM);
    cudaFuncSetAttribute(slab_kernel<float, 2>(), cudaFuncAttributeMaxDynamicSharedMemorySize, SLAB_MAX_SMEM);
    cudaFuncSetAttribute(slab_kernel<double, 2>(), cudaFuncAttributeMaxDynamicSharedMemorySize, SLAB_MAX_SMEM);
}

template <typename T>
cudaError_t launch_rb_slab(const LevelT<T>& L, const T* uin, T* uout, const T* b, int first, int zero_in,
                           const SlabShape& sh, cudaStream_t s)
{
    if (!slab_shape_ok(sh, sizeof(T)) || uin == uout || L.lsh) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((L.nx + sh.tx - 1) / sh.tx), (unsigned)((L.ny + sh.ty - 1) / sh.ty),
                    (unsigned)((L.nz + sh.kz - 1) / sh.kz));
    const size_t smem = slab_smem_bytes(sh, sizeof(T));
    if (sh.ns == 1)
        k_rb_col<T><<<grid, dim3(COL_PX, sh.ty + 2), smem, s>>>(L, uin, uout, b, first & 1, zero_in, sh.kz);
    else
        k_rb_slab<T, 2><<<grid, SLAB_NT, smem, s>>>(L, uin, uout, b, first & 1, zero_in, sh.tx, sh.ty, sh.kz);
    return cudaGetLastError();
}

template cudaError_t launch_rb_slab<float>(const LevelT<float>&, const float*, float*, const float*, int, int,
                                           const SlabShape&, cudaStream_t);
template cudaError_t launch_rb_slab<double>(const LevelT<double>&, const double*, double*, const double*, int, int,
                                            const SlabShape&, cudaStream_t);

}  // namespace lasto
