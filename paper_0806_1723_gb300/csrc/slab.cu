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
                        pc[o] = acc / (-(L.ax[0].dg[i] + L.ax[1].dg[j] + L.ax[2].dg[q]));
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

// One full sweep per pass with the z column in registers.  Thread (px, py) owns the node
// pair (i0 - 1 + 2 px, i0 + 2 px) of row j0 - 1 + py: one red and one black node in every
// plane.  The block covers the tile widened by one node (tx = 2 (PX - 1), ty = RY - 2).  At
// step p it updates the red node of plane p-1 (x/y neighbours from shared plane A: the old
// values; the edge threads bring one more node of halo), the black node of plane p-2 (x/y
// neighbours from shared plane B: the red values published a step earlier), and writes
// plane p-2.  Its pair's u and b for planes p-3 .. p+CD are a register ring that the loop,
// unrolled over the ring length, indexes with constants, so the loads of plane p+CD are in
// flight for CD steps; the halo arrives by cp.async into a ring of A planes.  B is
// double-buffered by step parity, so one barrier per step orders every shared read after
// its write.
constexpr int CD = 2;            // planes of prefetch
constexpr int CR = CD + 4;       // register ring: planes p-3 .. p+CD
constexpr int CWA = CD + 3;      // shared A ring

template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512)
    k_rb_col(LevelT<T> L, const T* __restrict__ uin, T* __restrict__ uout, const T* __restrict__ b, int first,
             int zero_in, int kz)
{
    extern __shared__ __align__(16) unsigned char col_smem[];
    const int PX = blockDim.x, RY = blockDim.y;
    const int TX = 2 * (PX - 1), TY = RY - 2;
    const int AX = TX + 4, AY = TY + 4, BX = TX + 2, AP = AX * AY;
    T* SA = reinterpret_cast<T*>(col_smem);           // [CWA][AY][AX]
    T* SB = SA + CWA * AP;                             // [2][RY][BX]
    T* ZC = SB + 2 * RY * BX;                          // [kz + 4][3]: cm, cp, dg of planes k0-2 ..
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int px = threadIdx.x, py = threadIdx.y, tid = py * PX + px, nth = PX * RY;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * kz;
    const int k1 = min(k0 + kz, nz);
    const int ia = i0 - 1 + 2 * px, j = j0 - 1 + py;
    const size_t sy = (size_t)nx, sz = (size_t)nx * ny;
    const bool row_in = j >= 0 && j < ny;
    const bool in_a = row_in && ia >= 0 && ia < nx, in_b = row_in && ia + 1 >= 0 && ia + 1 < nx;
    const bool row_int = j >= 1 && j <= ny - 2;
    const bool int_a = row_int && ia >= 1 && ia <= nx - 2, int_b = row_int && ia + 1 >= 1 && ia + 1 <= nx - 2;
    const bool row_tile = py >= 1 && py <= TY;
    const bool tile_a = row_tile && px >= 1, tile_b = row_tile && px <= PX - 2;
    const int oA = (py + 1) * AX + 2 * px + 1, oB = py * BX + 2 * px;

    for (int e = tid; e < kz + 4; e += nth) {
        const int qc = min(max(k0 - 2 + e, 0), nz - 1);
        ZC[3 * e] = L.ax[2].cm[qc];
        ZC[3 * e + 1] = L.ax[2].cp[qc];
        ZC[3 * e + 2] = L.ax[2].dg[qc];
    }
    const int ca = min(max(ia, 0), nx - 1), cb = min(max(ia + 1, 0), nx - 1), cj = min(max(j, 0), ny - 1);
    const T cmxa = L.ax[0].cm[ca], cpxa = L.ax[0].cp[ca], cmxb = L.ax[0].cm[cb], cpxb = L.ax[0].cp[cb];
    const T dga = L.ax[0].dg[ca], dgb = L.ax[0].dg[cb];
    const T cmy = L.ax[1].cm[cj], cpy = L.ax[1].cp[cj], dgy = L.ax[1].dg[cj];

    // halo of plane q into its A slot: the edge threads' nodes one step outside the block
    auto halo = [&](int q) {
        if (q < 0 || q >= nz) return;
        T* A = SA + ((q % CWA) + CWA) % CWA * AP;
        const size_t base = (size_t)q * sz;
        auto put = [&](int o, int jj, int ii) {
            if (jj < 0 || jj >= ny || ii < 0 || ii >= nx) return;
            if (zero_in)
                A[o] = T(0);
            else
                cp_async(A + o, uin + base + (size_t)jj * sy + ii);
        };
        if (px == 0) put((py + 1) * AX, j, i0 - 2);
        if (px == PX - 1) put((py + 1) * AX + AX - 1, j, i0 + TX + 1);
        if (py == 0) {
            put(2 * px + 1, j0 - 2, ia);
            put(2 * px + 2, j0 - 2, ia + 1);
        }
        if (py == RY - 1) {
            put((AY - 1) * AX + 2 * px + 1, j0 + TY + 1, ia);
            put((AY - 1) * AX + 2 * px + 2, j0 + TY + 1, ia + 1);
        }
    };
    auto ldu = [&](bool ok, int q, int ii) -> T {
        return (ok && !zero_in && q >= 0 && q < nz) ? uin[(size_t)q * sz + (size_t)j * sy + ii] : T(0);
    };
    auto ldb = [&](bool ok, int q, int ii) -> T {
        return (ok && q >= 1 && q <= nz - 2) ? b[(size_t)q * sz + (size_t)j * sy + ii] : T(0);
    };
    auto ldi = [&](bool ok, int q, int ii) -> T {
        if constexpr (sizeof(T) == 8)
            return (ok && q >= 1 && q <= nz - 2) ? L.inv_diag[(size_t)q * sz + (size_t)j * sy + ii] : T(0);
        return T(0);
    };

    // ring slot r holds plane p - 3 + ((r - s) mod CR) at unrolled step s
    T ua[CR], ub[CR], ba[CR], bb[CR], va[CR], vb[CR];
#pragma unroll
    for (int r = 0; r < CR; r++) {
        ua[r] = ub[r] = ba[r] = bb[r] = va[r] = vb[r] = T(0);
    }
    // prologue: planes k0-3 .. k0+CD-1 (ring slots 0 .. CR-2); halo of planes k0-1 .. k0+CD-1
#pragma unroll
    for (int r = 0; r < CR - 1; r++) {
        const int q = k0 - 3 + r;
        ua[r] = ldu(in_a, q, ia);
        ub[r] = ldu(in_b, q, ia + 1);
        ba[r] = ldb(int_a, q, ia);
        bb[r] = ldb(int_b, q, ia + 1);
        va[r] = ldi(int_a, q, ia);
        vb[r] = ldi(int_b, q, ia + 1);
    }
    for (int q = k0 - 1; q <= k0 + CD - 1; q++) {
        halo(q);
        cp_async_commit();
    }

    for (int p0 = k0; p0 <= k1 + 1; p0 += CR) {
#pragma unroll
        for (int s = 0; s < CR; s++) {
            const int p = p0 + s;
            if (p > k1 + 1) break;
            // ring slots of planes p-3 .. p+CD at this unrolled step
            const int r3 = (s + 0) % CR, r2 = (s + 1) % CR, r1 = (s + 2) % CR, r0 = (s + 3) % CR,
                      rn = (s + CR - 1) % CR;
            // loads of plane p + CD
            ua[rn] = ldu(in_a, p + CD, ia);
            ub[rn] = ldu(in_b, p + CD, ia + 1);
            ba[rn] = ldb(int_a, p + CD, ia);
            bb[rn] = ldb(int_b, p + CD, ia + 1);
            va[rn] = ldi(int_a, p + CD, ia);
            vb[rn] = ldi(int_b, p + CD, ia + 1);
            halo(p + CD);
            cp_async_commit();
            // publish plane p-1 (old values; the halo is already on its way into the slot)
            T* A = SA + (((p - 1) % CWA) + CWA) % CWA * AP;
            A[oA] = ua[r1];
            A[oA + 1] = ub[r1];
            asm volatile("cp.async.wait_group %0;\n" ::"n"(CD + 1) : "memory");
            __syncthreads();
            const T* Bp = SB + ((p - 1) & 1) * RY * BX;
            T* Bn = SB + (p & 1) * RY * BX;
            // red node of plane q = p - 1
            const int q = p - 1;
            if (q >= max(1, k0 - 1) && q <= min(nz - 2, k1)) {
                const T* zc = ZC + 3 * (q - k0 + 2);
                const bool red_a = ((ia + j + q) & 1) == first;
                if (red_a ? int_a : int_b) {
                    const int o = red_a ? oA : oA + 1;
                    const T xm = red_a ? A[o - 1] : ua[r1];
                    const T xp = red_a ? ub[r1] : A[o + 1];
                    T t = (red_a ? cmxa : cmxb) * xm;
                    t = fma(red_a ? cpxa : cpxb, xp, t);
                    t = fma(cmy, A[o - AX], t);
                    t = fma(cpy, A[o + AX], t);
                    t = fma(zc[0], red_a ? ua[r2] : ub[r2], t);
                    t = fma(zc[1], red_a ? ua[r0] : ub[r0], t);
                    const T acc = (red_a ? ba[r1] : bb[r1]) - t;
                    T v;
                    if constexpr (sizeof(T) == 8)
                        v = acc * (red_a ? va[r1] : vb[r1]);
                    else
                        v = acc / (-((red_a ? dga : dgb) + dgy + zc[2]));
                    if (red_a)
                        ua[r1] = v;
                    else
                        ub[r1] = v;
                }
            }
            // black node of plane q2 = p - 2 (tile nodes only)
            const int q2 = p - 2;
            if (q2 >= max(1, k0) && q2 <= min(nz - 2, k1 - 1)) {
                const T* zc = ZC + 3 * (q2 - k0 + 2);
                const bool blk_a = ((ia + j + q2) & 1) != first;
                if (blk_a ? (int_a && tile_a) : (int_b && tile_b)) {
                    const int o = blk_a ? oB : oB + 1;
                    const T xm = blk_a ? Bp[o - 1] : ua[r2];
                    const T xp = blk_a ? ub[r2] : Bp[o + 1];
                    T t = (blk_a ? cmxa : cmxb) * xm;
                    t = fma(blk_a ? cpxa : cpxb, xp, t);
                    t = fma(cmy, Bp[o - BX], t);
                    t = fma(cpy, Bp[o + BX], t);
                    t = fma(zc[0], blk_a ? ua[r3] : ub[r3], t);
                    t = fma(zc[1], blk_a ? ua[r1] : ub[r1], t);
                    const T acc = (blk_a ? ba[r2] : bb[r2]) - t;
                    T v;
                    if constexpr (sizeof(T) == 8)
                        v = acc * (blk_a ? va[r2] : vb[r2]);
                    else
                        v = acc / (-((blk_a ? dga : dgb) + dgy + zc[2]));
                    if (blk_a)
                        ua[r2] = v;
                    else
                        ub[r2] = v;
                }
            }
            if (q2 >= k0 && q2 < k1) {
                const size_t P = (size_t)q2 * sz + (size_t)j * sy + ia;
                if (in_a && tile_a) uout[P] = ua[r2];
                if (in_b && tile_b) uout[P + 1] = ub[r2];
            }
            // publish the red values of plane p-1 for the next step's black update
            Bn[oB] = ua[r1];
            Bn[oB + 1] = ub[r1];
        }
    }
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

// ns = 1 runs the column kernel (block (tx/2 + 1) x (ty + 2) threads); ns = 2 the z-slab
// window kernel (256 threads).
size_t slab_smem_bytes(const SlabShape& sh, size_t elem)
{
    if (sh.ns == 1) {
        const size_t AX = sh.tx + 4, AY = sh.ty + 4, BX = sh.tx + 2, RY = sh.ty + 2;
        return (CWA * AX * AY + 2 * RY * BX + 3 * ((size_t)sh.kz + 4)) * elem;
    }
    const size_t H = 2 * (size_t)sh.ns;
    return (2 * (size_t)sh.ns + 3) * ((size_t)sh.tx + 2 * H) * ((size_t)sh.ty + 2 * H) * elem;
}

bool slab_shape_ok(const SlabShape& sh, size_t elem)
{
    if (sh.ns == 1)
        return sh.tx >= 2 && sh.tx % 2 == 0 && sh.ty >= 1 && sh.kz >= 1 && sh.kz <= 4096 &&
               (sh.tx / 2 + 1) * (sh.ty + 2) <= (elem == 8 ? 256 : 512) && slab_smem_bytes(sh, elem) <= SLAB_MAX_SMEM;
    return sh.ns == 2 && sh.tx >= 2 && sh.ty >= 1 && sh.kz >= 1 && sh.tx <= 512 && sh.ty <= 512 &&
           slab_smem_bytes(sh, elem) <= SLAB_MAX_SMEM;
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
    if (!slab_shape_ok(sh, sizeof(T)) || uin == uout) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((L.nx + sh.tx - 1) / sh.tx), (unsigned)((L.ny + sh.ty - 1) / sh.ty),
                    (unsigned)((L.nz + sh.kz - 1) / sh.kz));
    const size_t smem = slab_smem_bytes(sh, sizeof(T));
    if (sh.ns == 1)
        k_rb_col<T><<<grid, dim3(sh.tx / 2 + 1, sh.ty + 2), smem, s>>>(L, uin, uout, b, first & 1, zero_in, sh.kz);
    else
        k_rb_slab<T, 2><<<grid, SLAB_NT, smem, s>>>(L, uin, uout, b, first & 1, zero_in, sh.tx, sh.ty, sh.kz);
    return cudaGetLastError();
}

template cudaError_t launch_rb_slab<float>(const LevelT<float>&, const float*, float*, const float*, int, int,
                                           const SlabShape&, cudaStream_t);
template cudaError_t launch_rb_slab<double>(const LevelT<double>&, const double*, double*, const double*, int, int,
                                            const SlabShape&, cudaStream_t);

}  // namespace lasto
