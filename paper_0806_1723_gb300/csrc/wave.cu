// Fused red-black Gauss-Seidel sweep, one full sweep per pass, as a z wavefront over row
// chunks staged in shared memory (Section 3: the finite-difference multigrid smoother).
//
// One pass reads u_in and b once and writes u_out once (12 bytes per node in FP32), where
// two in-place half-sweep launches stream the grid twice.  A CTA owns a tile of tx columns
// and TY rows of the (x, y) plane and walks a range of z.  At step k it updates the first
// colour of plane k+1 (stage 1: the other colour's old values are its neighbours) and then
// the second colour of plane k (stage 2: the first colour's new values, planes k-1..k+1, are
// its neighbours), so the sweep equals the in-place pair of half sweeps bit for bit: every
// node update is the in-place kernels' expression with the same operands.  Stage 1 also
// covers one ring of nodes around the tile (rows j0-1 and j0+TY, columns x0-1 and x0+tx) and
// the two planes before the z range, which the neighbouring CTAs compute too, with the same
// operands and arithmetic.
//
// Layout.  Grids have an odd number of nodes per axis, so the parity of the flat index is
// the colour.  Each lane owns a pair of nodes (P, P+1) with P even: the first of every pair
// is colour 0, the second colour 1, in every row and plane.  The pairs of a row start at
// floor2(a - 1), a = flat index of the tile's first column in that row; 32 lanes cover 64
// flat indices, enough for the tile (tx <= 60) and its ring.  The row's chunk in shared
// memory starts at floor4 of that minus one and holds 72 values (eighteen 16-byte aligned
// pieces), which covers every x, y and z neighbour of the pairs.  With m = a mod 4 the pair
// sits at chunk offset C0(m) = (2, 4, 4, 2) and the chunk starts at a - D(m), D = (4, 5, 6,
// 3); a neighbour row or plane (tile start a + delta) is read at the node's own offset plus
// D((m + delta) mod 4) - D(m), which depends on m and delta mod 4 only: four small tables per
// level, looked up with one byte permute.  Rows and planes outside the grid are not copied;
// no update or output reads them.
//
// Pipeline.  Group G of a unit copies u plane k_first + G (TY + 4 rows) and b plane
// k_first + G - 1 (TY + 2 rows) into ring slot G mod 8, as 16-byte cp.async pieces spread
// over the whole block (one commit group per G).  Step t waits until groups up to t + 2 have
// landed, passes the block's one barrier of the step, and then issues group t + 6 into the
// slot of group t - 2 (whose last reader, step t - 1, is behind that barrier).  The step
// loop is unrolled by the ring length, so slot offsets are constants.  The waits are the
// hardware's own (no spin), and every copy reads inside the array, so no wait can outlast
// the copies.
//
// Work split.  A unit is one tile and one of Z equal z ranges; units are numbered z-range
// major and dealt round robin to the resident CTAs, so neighbouring tiles walk the same
// planes at the same time and the rows they share are read from L2.  Z is chosen on the
// host so that the units fill whole waves of resident CTAs.
#include <algorithm>
#include <type_traits>

#include "internal.cuh"

namespace lasto {

namespace {

constexpr int WV_PITCH = 72;                         // values per staged row chunk

__device__ __forceinline__ uint32_t wv_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__host__ __device__ __forceinline__ int wv_D(int m) { return (0x3654 >> (4 * m)) & 15; }

// byte m of a four-entry table (zero-extended), m = 0..3
__device__ __forceinline__ uint32_t wv_pick(uint32_t table, uint32_t sel) { return __byte_perm(table, 0u, sel); }

struct WaveArgs {
    LevelT<float> L;
    const float* uin;
    float* uout;
    const float* b;
    int tx;
    int nzc;                  // z ranges per tile (units = tiles x nzc)
    // byte m of each word, m = 0..3: D(m); 4 C0(m); and 4 (D(m') - D(m)) + 32 for the neighbour
    // in row j-1, row j+1, plane p-1, plane p+1 (m' = (m + delta) mod 4)
    uint32_t tD, tC0, tym, typ, tzm, tzp;
};

constexpr int WV_ZMAX = 256;   // planes per unit (+ 3) the z-coefficient table holds

template <int TY, int S, int FIRST>
__global__ void __launch_bounds__(32 * (TY + 2), TY >= 12 ? 2 : 3) k_rb_wave(const WaveArgs A)
{
    constexpr int NT = 32 * (TY + 2);
    constexpr int UROWS = TY + 4, BROWS = TY + 2;
    constexpr uint32_t ROWB = WV_PITCH * 4;                      // bytes per staged row
    constexpr uint32_t USLOTB = UROWS * ROWB, BSLOTB = BROWS * ROWB;
    constexpr int CPR = WV_PITCH / 4;                            // 16-byte pieces per row
    constexpr int NCHUNK = (UROWS + BROWS) * CPR;                // per group
    constexpr int NSECOND = NCHUNK - NT;                         // threads with a second piece
    constexpr int D = S - 4;                                     // groups in flight beyond the live window
    constexpr uint32_t E1 = FIRST, E2 = 1 - FIRST;               // pair element of stage 1 / stage 2
    static_assert(S == 8 && NSECOND > 0 && NSECOND <= NT && UROWS * CPR <= NT, "ring and copy split");
    extern __shared__ __align__(128) unsigned char wv_smem_raw[];
    constexpr uint32_t SU = 0, SB = S * USLOTB, SZ = SB + S * BSLOTB;   // u ring, b ring, z table
    auto F = [&](uint32_t off) -> float& { return *reinterpret_cast<float*>(wv_smem_raw + off); };
    const uint32_t smem_base = wv_smem(wv_smem_raw);

    const LevelT<float>& L = A.L;
    const int nx = L.nx, ny = L.ny, nz = L.nz, tx = A.tx;
    const int nxny = nx * ny;
    const int N = nxny * nz;
    const int dZ = nxny & 3;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntx = (nx + tx - 1) / tx, nty = (ny + TY - 1) / TY;
    const int ntiles = ntx * nty, units = ntiles * A.nzc;

    for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
        const int zc = unit / ntiles, tile = unit - zc * ntiles;
        const int k0 = (int)((long long)nz * zc / A.nzc), k1 = (int)((long long)nz * (zc + 1) / A.nzc);
        const int x0 = (tile % ntx) * tx, j0 = (tile / ntx) * TY;
        const int xend = min(x0 + tx, nx);
        const int kf = k0 - 2;                 // step t works on k = kf + t
        const int nsteps = k1 - kf;            // k = k0-2 .. k1-1
        const int ngroups = nsteps + 2;        // group G (slot G mod 8): u plane kf + G, b plane kf + G - 1

        // every copy of the previous unit has landed and every read of it is done (its last
        // step's barrier), so the ring restarts at slot 0 and the z table is free
        __syncthreads();
        for (int e = threadIdx.x; e <= nsteps; e += NT) {   // z coefficients, entry t = plane kf + t
            const int q = kf + e;
            const bool in = q >= 0 && q < nz;
            F(SZ + 12u * e) = in ? L.ax[2].cm[q] : 0.0f;
            F(SZ + 12u * e + 4) = in ? L.ax[2].cp[q] : 0.0f;
            F(SZ + 12u * e + 8) = in ? L.ax[2].dg[q] : 0.0f;
        }

        // ---- this thread's pieces of every group: piece 0 (every thread; a u piece for the
        // first UROWS * CPR threads, else a b piece) and piece 1 (threads below NSECOND; a b
        // piece).  Per piece: its row's tile-start index a at the next group to issue (a grows
        // by nx*ny per group), its chunk column, its destination in slot 0, its plane.
        int ca[2], cc[2], cpl[2];
        uint32_t cdst[2];
        bool crow[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int q = threadIdx.x + h * NT;
            const bool isu = q < UROWS * CPR;
            const int qq = isu ? q : q - UROWS * CPR;
            const int r = qq / CPR, c = qq - r * CPR;
            const int j = isu ? j0 - 2 + r : j0 - 1 + r;
            cc[h] = 4 * c;
            cpl[h] = isu ? kf : kf - 1;
            ca[h] = (cpl[h] * ny + j) * nx + x0;
            crow[h] = q < NCHUNK && j >= 0 && j < ny;
            cdst[h] = smem_base + (isu ? SU + r * ROWB : SB + r * ROWB) + 16 * c;
        }
        const bool u0 = threadIdx.x < UROWS * CPR;
        const float* src0 = u0 ? A.uin : A.b;
        const uint32_t stride0 = u0 ? USLOTB : BSLOTB;
        // group G into slot G mod 8, as 16-byte cp.async pieces over the whole block, one
        // commit per group (empty beyond the unit, so that wait_group counts stay uniform).  A
        // piece reaching past the array's end copies its valid bytes and zero-fills the rest;
        // pieces before the array's start, or in rows and planes outside the grid, are not
        // copied (nothing reads them).  Groups are issued in order.
        auto piece = [&](int h, uint32_t so) {
            const int a = ca[h];
            const int e = a + cc[h] - (int)wv_pick(A.tD, 0x4440u | (uint32_t)(a & 3));   // first element
            if (crow[h] && (unsigned)cpl[h] < (unsigned)nz && (unsigned)e < (unsigned)N) {
                const int bytes = min(16, 4 * (N - e));
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(
                                 cdst[h] + so * (h == 0 ? stride0 : BSLOTB)),
                             "l"((h == 0 ? src0 : A.b) + e), "r"(bytes));
            }
            ca[h] = a + nxny;
            cpl[h] += 1;
        };
        auto issue = [&](int G) {
            if (G < ngroups) {
                const uint32_t so = (uint32_t)(G & (S - 1));
                piece(0, so);
                if (warp < (NSECOND + 31) / 32) piece(1, so);
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        };
        for (int G = 0; G < D + 2; G++) issue(G);

        // ---- this warp's row, and per lane the coefficients of its two nodes for the parity
        // of m at even steps (index 0) and at odd steps (index 1): m changes parity every plane
        const int j = j0 - 1 + warp;
        const int jc = min(max(j, 0), ny - 1);
        const float cmy = L.ax[1].cm[jc], cpy = L.ax[1].cp[jc], dgy = L.ax[1].dg[jc];
        const bool row_int = j >= 1 && j <= ny - 2;
        const bool row_tile = warp >= 1 && warp <= TY && j < ny;
        const int m_first = (((kf + 1) * ny + j) * nx + x0) & 3;   // m of this row at plane k+1 of step 0
        const int par0 = m_first & 1;
        float cm1[2], cp1[2], dg1[2], cm2[2], cp2[2], dg2[2];
        // bits (q): 0+ stage-1 update, 2+ stage-2 update, 4+ write first node, 6+ write second
        uint32_t fl = 0;
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int par = par0 ^ q;
            const int xl = x0 - 2 + par + 2 * lane;            // column of the pair's first node
            const int x1 = xl + (int)E1, x2 = xl + (int)E2;
            const int c1 = min(max(x1, 0), nx - 1), c2 = min(max(x2, 0), nx - 1);
            cm1[q] = L.ax[0].cm[c1];
            cp1[q] = L.ax[0].cp[c1];
            dg1[q] = L.ax[0].dg[c1] + dgy;                     // (dgx + dgy) + dgz, as the in-place sweep
            cm2[q] = L.ax[0].cm[c2];
            cp2[q] = L.ax[0].cp[c2];
            dg2[q] = L.ax[0].dg[c2] + dgy;
            fl |= (uint32_t)(row_int && x1 >= 1 && x1 <= nx - 2) << q;
            fl |= (uint32_t)(row_int && row_tile && x2 >= x0 && x2 < xend && x2 >= 1 && x2 <= nx - 2) << (2 + q);
            fl |= (uint32_t)(row_tile && xl >= x0 && xl < xend) << (4 + q);
            fl |= (uint32_t)(row_tile && xl + 1 >= x0 && xl + 1 < xend) << (6 + q);
        }
        const uint32_t lane_b = 8u * lane;
        const uint32_t ru_b = (uint32_t)(warp + 1) * ROWB, rb_b = (uint32_t)warp * ROWB;
        // first node of the lane's pair at plane k of step 0, for parity 0 of m
        float* outp = A.uout + ((kf * ny + j) * nx + x0 - 2 + 2 * lane);
        float zc0 = 0.0f, zc1 = 0.0f, zc2 = 0.0f;            // plane k coefficients (read a step earlier)

        // step t = T0 + TT, TT = t mod 8 known: ring slots and the parity index are constants
        auto step = [&](int t, auto ttc) {
            constexpr int TT = decltype(ttc)::value;
            constexpr int Q1 = TT & 1, Q2 = 1 - Q1;
            constexpr uint32_t Um = SU + ((TT + 7) & 7) * USLOTB, U0 = SU + (TT & 7) * USLOTB;
            constexpr uint32_t U1 = SU + ((TT + 1) & 7) * USLOTB, U2 = SU + ((TT + 2) & 7) * USLOTB;
            constexpr uint32_t B0 = SB + ((TT + 1) & 7) * BSLOTB, B1 = SB + ((TT + 2) & 7) * BSLOTB;
            const int k = kf + t;
            // groups <= t + 2 have landed (t + 1 + D is the newest issued), every thread's copies
            // are visible, and step t - 1 is done: its reads of the slot of group t - 2 and its
            // stage-1 writes of plane k
            asm volatile("cp.async.wait_group %0;\n" ::"n"(D - 1) : "memory");
            __syncthreads();
            issue(t + 2 + D);   // into the slot of group t - 2

            // ---------------- stage 1: first colour of plane p = k + 1
            const int p = k + 1;
            const uint32_t zt = SZ + 12u * (uint32_t)(t + 1);
            const float zn0 = F(zt), zn1 = F(zt + 4), zn2 = F(zt + 8);
            if (p >= 1 && p <= nz - 2 && ((fl >> Q1) & 1u)) {
                const uint32_t sel = 0x4440u | (uint32_t)((m_first + TT * dZ) & 3);   // m at plane k+1
                const uint32_t o = wv_pick(A.tC0, sel) + 4u * E1 + lane_b + ru_b;
                float t1 = cm1[Q1] * F(U1 + o - 4);
                t1 = fmaf(cp1[Q1], F(U1 + o + 4), t1);
                t1 = fmaf(cmy, F(U1 + o + wv_pick(A.tym, sel) - ROWB - 32), t1);
                t1 = fmaf(cpy, F(U1 + o + wv_pick(A.typ, sel) + ROWB - 32), t1);
                t1 = fmaf(zn0, F(U0 + o + wv_pick(A.tzm, sel) - 32), t1);
                t1 = fmaf(zn1, F(U2 + o + wv_pick(A.tzp, sel) - 32), t1);
                const float acc = F(B1 - ru_b + rb_b + o) - t1;
                F(U1 + o) = rb_point32(acc, dg1[Q1] + zn2);
            }
            __syncwarp();
            // ---------------- stage 2: second colour of plane k, then the plane's tile is final
            if (t >= 2 && row_tile) {
                const uint32_t sel = 0x4440u | (uint32_t)((m_first + (TT + 3) * dZ) & 3);   // m at plane k
                const uint32_t op = wv_pick(A.tC0, sel) + lane_b + ru_b;   // the lane's pair
                const float2 pr = *reinterpret_cast<const float2*>(wv_smem_raw + U0 + op);
                float v0 = pr.x, v1 = pr.y;
                if (k >= 1 && k <= nz - 2 && ((fl >> (2 + Q2)) & 1u)) {
                    const uint32_t o = op + 4u * E2;
                    const float xm = E2 ? v0 : F(U0 + o - 4);
                    const float xp = E2 ? F(U0 + o + 4) : v1;
                    float t2 = cm2[Q2] * xm;
                    t2 = fmaf(cp2[Q2], xp, t2);
                    t2 = fmaf(cmy, F(U0 + o + wv_pick(A.tym, sel) - ROWB - 32), t2);
                    t2 = fmaf(cpy, F(U0 + o + wv_pick(A.typ, sel) + ROWB - 32), t2);
                    t2 = fmaf(zc0, F(Um + o + wv_pick(A.tzm, sel) - 32), t2);
                    t2 = fmaf(zc1, F(U1 + o + wv_pick(A.tzp, sel) - 32), t2);
                    const float acc = F(B0 - ru_b + rb_b + o) - t2;
                    const float nv = rb_point32(acc, dg2[Q2] + zc2);
                    if (E2) v1 = nv; else v0 = nv;
                }
                const bool il = (fl >> (4 + Q2)) & 1u, ir = (fl >> (6 + Q2)) & 1u;
                float* out = outp + (par0 ^ Q2);
                if (il && ir)
                    *reinterpret_cast<float2*>(out) = make_float2(v0, v1);
                else if (il)
                    out[0] = v0;
                else if (ir)
                    out[1] = v1;
            }
            outp += nxny;
            zc0 = zn0;
            zc1 = zn1;
            zc2 = zn2;
        };
        using std::integral_constant;
        for (int t = 0; t < nsteps; t += 8) {
            step(t, integral_constant<int, 0>{});
            if (t + 1 < nsteps) step(t + 1, integral_constant<int, 1>{});
            if (t + 2 < nsteps) step(t + 2, integral_constant<int, 2>{});
            if (t + 3 < nsteps) step(t + 3, integral_constant<int, 3>{});
            if (t + 4 < nsteps) step(t + 4, integral_constant<int, 4>{});
            if (t + 5 < nsteps) step(t + 5, integral_constant<int, 5>{});
            if (t + 6 < nsteps) step(t + 6, integral_constant<int, 6>{});
            if (t + 7 < nsteps) step(t + 7, integral_constant<int, 7>{});
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}


template <int TY, int S>
size_t wave_smem()
{
    return sizeof(float) * ((size_t)S * ((TY + 4) + (TY + 2)) * WV_PITCH + 3 * WV_ZMAX);
}

template <int TY, int S, int FIRST>
void* wave_kernel()
{
    return reinterpret_cast<void*>(&k_rb_wave<TY, S, FIRST>);
}

// Occupancy-sized grid of one instantiation on the current device (cached per device).
template <int TY, int S, int FIRST>
int wave_resident_ctas()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (cached[dev] > 0) return cached[dev];
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rb_wave<TY, S, FIRST>, 32 * (TY + 2),
                                                      wave_smem<TY, S>()) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
        return 0;
    cached[dev] = per_sm * sms;
    return cached[dev];
}

template <int TY, int S, int FIRST>
cudaError_t launch_wave_t(WaveArgs a, cudaStream_t s)
{
    const int ctas = wave_resident_ctas<TY, S, FIRST>();
    if (ctas < 1) return cudaErrorInvalidConfiguration;
    const int nx = a.L.nx, ny = a.L.ny, nz = a.L.nz;
    const long long tiles = (long long)((nx + a.tx - 1) / a.tx) * ((ny + TY - 1) / TY);
    // z ranges per tile: fill whole waves of resident CTAs, each range paying two extra planes
    double best = 1e30;
    a.nzc = (nz + WV_ZMAX - 4) / (WV_ZMAX - 3);
    for (int zc = 1; zc <= std::min(64, nz); zc++) {
        if ((nz + zc - 1) / zc + 3 > WV_ZMAX) continue;   // the unit's planes fit the z table
        const long long units = tiles * zc;
        const double waves = (double)((units + ctas - 1) / ctas);
        const double cost = waves * (nz / (double)zc + 2.0);   // steps of the busiest CTA
        if (cost < best * (1.0 - 1e-9)) {
            best = cost;
            a.nzc = zc;
        }
    }
    const long long units = tiles * a.nzc;
    const int grid = (int)std::min<long long>(units, ctas);
    k_rb_wave<TY, S, FIRST><<<grid, 32 * (TY + 2), wave_smem<TY, S>(), s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool wave_shape_ok(const SlabShape& sh)
{
    return sh.ns == 1 && sh.tx >= 16 && sh.tx <= 60 && (sh.ty == 8 || sh.ty == 12 || sh.ty == 16) && sh.kz == 8;
}

bool wave_level_ok(int nx, int ny, int nz)
{
    // with rows of at least 69 nodes every chunk lies inside the array except in the first row
    // of the first plane and the last row of the last plane (copied in part)
    // (the tile-start index of the planes just past the grid stays below 2^31 too)
    return nx >= 69 && ny >= 3 && nz >= 3 && (size_t)nx * ny * ((size_t)nz + 4) < (size_t(1) << 31);
}

void init_wave_attributes()
{
    cudaFuncSetAttribute(wave_kernel<16, 8, 0>(), cudaFuncAttributeMaxDynamicSharedMemorySize, wave_smem<16, 8>());
    cudaFuncSetAttribute(wave_kernel<16, 8, 1>(), cudaFuncAttributeMaxDynamicSharedMemorySize, wave_smem<16, 8>());
    cudaFuncSetAttribute(wave_kernel<12, 8, 0>(), cudaFuncAttributeMaxDynamicSharedMemorySize, wave_smem<12, 8>());
    cudaFuncSetAttribute(wave_kernel<12, 8, 1>(), cudaFuncAttributeMaxDynamicSharedMemorySize, wave_smem<12, 8>());
    cudaFuncSetAttribute(wave_kernel<8, 8, 0>(), cudaFuncAttributeMaxDynamicSharedMemorySize, wave_smem<8, 8>());
    cudaFuncSetAttribute(wave_kernel<8, 8, 1>(), cudaFuncAttributeMaxDynamicSharedMemorySize, wave_smem<8, 8>());
}

cudaError_t launch_rb_wave(const LevelT<float>& L, const float* uin, float* uout, const float* b, int first,
                           const SlabShape& sh, cudaStream_t s)
{
    if (!wave_shape_ok(sh) || !wave_level_ok(L.nx, L.ny, L.nz) || uin == uout || L.lsh) return cudaErrorInvalidValue;
    // 16-byte aligned arrays: the staged copies read 16-byte aligned chunks
    if ((reinterpret_cast<uintptr_t>(uin) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(uout)) & 15)
        return cudaErrorInvalidValue;
    WaveArgs a{L, uin, uout, b, sh.tx, 1, 0u, 0u, 0u, 0u, 0u, 0u};
    const int nx = L.nx, nxny = L.nx * L.ny;
    const int deltas[4] = {-nx, nx, -nxny, nxny};
    uint32_t* words[4] = {&a.tym, &a.typ, &a.tzm, &a.tzp};
    for (int m = 0; m < 4; m++) {
        a.tD |= (uint32_t)wv_D(m) << (8 * m);
        a.tC0 |= (uint32_t)(4 * ((0x2442 >> (4 * m)) & 15)) << (8 * m);
        for (int q = 0; q < 4; q++) {
            const int shift = wv_D(((m + deltas[q]) % 4 + 4) % 4) - wv_D(m);   // -3 .. 3 nodes
            *words[q] |= (uint32_t)(4 * shift + 32) << (8 * m);
        }
    }
    if (sh.ty == 16)
        return (first & 1) ? launch_wave_t<16, 8, 1>(a, s) : launch_wave_t<16, 8, 0>(a, s);
    if (sh.ty == 12)
        return (first & 1) ? launch_wave_t<12, 8, 1>(a, s) : launch_wave_t<12, 8, 0>(a, s);
    return (first & 1) ? launch_wave_t<8, 8, 1>(a, s) : launch_wave_t<8, 8, 0>(a, s);
}

}  // namespace lasto
