// The FP32 red-black half sweep over colour-split storage with its operands staged in shared
// memory by bulk copies (Section 3's smoother, the same node update as k_rbgs_split_rows).
//
// In colour-split storage the rows of one colour are consecutive, so the nodes a tile of R
// interior rows of plane k reads from the other colour -- its own rows and the rows j0 - 1 and
// j0 + R of planes k - 1, k, k + 1 -- are one contiguous run per plane, and the tile's own
// right-hand side is another.  A block owns R rows (one warp each) and a chunk of planes,
// marches through the chunk in z and keeps the other colour's planes k - 1, k, k + 1 in a ring
// of SG_NS slots with the next plane in flight (cp.async.bulk, completion counted on an
// mbarrier), the right-hand side in SG_NB slots.  Each plane of the other colour is read from
// DRAM once per (tile, chunk), and every warp's loads are shared-memory loads whose operands
// arrived a plane earlier: the row-per-warp kernel's loads wait on L2 and DRAM one row at a
// time.  Results go straight to global memory (the colour being written is not read in this
// half sweep).
//
// The same kernel forms the red residuals for the restriction (MODE 1) and the first red half
// sweep from a zero iterate (MODE 2); the file also holds the staged prolongation onto a
// colour-split level (k_prolong_stage), which stages the coarse rows the same way.
//
// Waits are bounded: a wait that runs out (about two seconds) raises LASTO_ERR_TIMEOUT in
// *status (when given), the block waits -- again bounded -- for the copies it has in flight and
// leaves.
#include "stage.cuh"

namespace lasto {

namespace {

using namespace stage;

constexpr int SG_R = 8;              // interior rows per tile, one warp each
constexpr int SG_NT = 32 * SG_R;
constexpr int SG_NS = 4;             // other-colour plane slots: k - 1, k, k + 1, one in flight
constexpr int SG_NB = 2;             // right-hand-side plane slots: k, one in flight

// MODE 0: the half sweep of `colour` in place on u.  MODE 1: no update; the residuals b - A u
// of the colour's nodes go to r at the nodes' own storage positions (the restriction after a
// black half sweep reads those of the red nodes: the black ones are then zero).  MODE 2: the
// half sweep of `colour` from an other colour that is zero: every neighbour term is +0, so the
// other colour is neither staged nor read (its stale values may be anything) and the result is
// bitwise the half sweep's over zeros.
template <int V, int MODE>
__global__ void __launch_bounds__(SG_NT) k_rbgs_split_stage(LevelT<float> L, float* __restrict__ u, const float* __restrict__ b,
                                                            int colour, StageGeom g, int* __restrict__ status,
                                                            float* __restrict__ r)
{
    constexpr bool RESID = MODE == 1, ZO = MODE == 2;
    extern __shared__ __align__(16) float sg[];
    __shared__ __align__(8) uint64_t bar_o[SG_NS];
    __shared__ __align__(8) uint64_t bar_b[SG_NB];
    __shared__ unsigned ost[SG_NS], bst[SG_NB];   // global start of each slot's run (thread 0 writes it
                                                  // before the copy's arrive; readers wait on the copy)
    float* so = sg;                          // [SG_NS][oslot]
    float* sb = sg + SG_NS * g.oslot;        // [SG_NB][bslot]
    float* sx = sb + SG_NB * g.bslot;        // x coefficients [2 parities][cm, cp, dg][g.hx1]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tj = (int)(blockIdx.x % (unsigned)g.tiles_j), kc = (int)(blockIdx.x / (unsigned)g.tiles_j);
    const int j0 = 1 + tj * SG_R;
    const int nr = min(SG_R, L.ny - 1 - j0);           // the tile's interior rows
    const int kA = 1 + kc * g.chunk, kB = min(L.nz - 2, kA + g.chunk - 1);
    if (nr <= 0 || kA > kB) return;
    const int c = colour;
    const int nx = L.nx;
    const unsigned nxy = (unsigned)nx * (unsigned)L.ny;
    const int hx = (nx - 1) >> 1, hxy = (int)((nxy - 1) >> 1);
    const int dxm = c - 1, dxp = c, dym = c - 1 - hx, dyp = c + hx, dzm = c - 1 - hxy, dzp = c + hxy;
    const int oLast = kB + 1, o0 = kA - 1;           // other-colour planes o0 .. oLast, in order
    // planes issued so far (thread 0's counts; the waits derive slot and parity from the plane)
    int o_next = o0, b_next = kA;
    if (tid == 0) {
        for (int q = 0; q < SG_NS; q++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sg_smem(&bar_o[q])) : "memory");
        for (int q = 0; q < SG_NB; q++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sg_smem(&bar_b[q])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // the x coefficients of the colour's interior nodes by parity of the first one (i1 = 1, 2):
    // node s of a run is i1 + 2 s; one copy per block, read conflict-free by consecutive lanes
    for (int t = tid; t < 2 * g.hx1; t += SG_NT) {
        const int par = t / g.hx1, sx_i = t - par * g.hx1;
        const int i = 1 + par + 2 * sx_i;
        const bool in = i < nx - 1;
        sx[(par * 3 + 0) * g.hx1 + sx_i] = in ? L.ax[0].cm[i] : 0.0f;
        sx[(par * 3 + 1) * g.hx1 + sx_i] = in ? L.ax[0].cp[i] : 0.0f;
        sx[(par * 3 + 2) * g.hx1 + sx_i] = in ? L.ax[0].dg[i] : 0.0f;
    }
    __syncthreads();
    if (tid == 0) {
        for (; !ZO && o_next <= oLast && o_next < o0 + SG_NS; o_next++) {
            unsigned st, ln;
            sg_orange(L, c, o_next, j0, nr, st, ln);
            const int q = (o_next - o0) % SG_NS;
            ost[q] = st;
            sg_issue(u, st, ln, so + q * g.oslot, sg_smem(&bar_o[q]));
        }
        for (; b_next <= kB && b_next < kA + SG_NB; b_next++) {
            unsigned st, ln;
            sg_brange(L, c, b_next, j0, nr, st, ln);
            const int q = (b_next - kA) % SG_NB;
            bst[q] = st;
            sg_issue(b, st, ln, sb + q * g.bslot, sg_smem(&bar_b[q]));
            if (RESID) sg_prefetch(u, st, ln);   // the colour's own values, read from global
        }
    }
    // the warp's row and its x coefficients (row-independent but for the colour's first node)
    const int j = j0 + warp;
    const bool has_row = warp < nr;
    const float cmy = has_row ? L.ax[1].cm[j] : 0.0f, cpy = has_row ? L.ax[1].cp[j] : 0.0f;
    const float dgy = has_row ? L.ax[1].dg[j] : 0.0f;
    bool failed = false;
    for (int k = kA; k <= kB; k++) {
        bool bad = false;
        {
            // planes k - 1 and k were waited for at the previous step (or here, at the first)
            for (int p = (k == kA ? k - 1 : k + 1); p <= k + 1 && !ZO; p++) {
                const int d = p - o0;
                if (!bad && !sg_wait(sg_smem(&bar_o[d % SG_NS]), (uint32_t)((d / SG_NS) & 1))) bad = true;
            }
            const int d = k - kA;
            if (!bad && !sg_wait(sg_smem(&bar_b[d % SG_NB]), (uint32_t)((d / SG_NB) & 1))) bad = true;
        }
        if (!bad && has_row) {
            const int i1 = ((c + j + k) & 1) ? 1 : 2;      // first interior node of the colour
            const int left = ((nx - i1) >> 1) - lane;
            const unsigned q0 = ((unsigned)k * nxy + (unsigned)j * (unsigned)nx + (unsigned)i1) >> 1;
            const unsigned go = (unsigned)(1 - c) * L.H + q0 + (unsigned)lane;   // lane's node, other colour
            const float* ok = ZO ? so : so + ((k - o0) % SG_NS) * g.oslot + (go - ost[(k - o0) % SG_NS]);
            const float* om = ZO ? so : so + ((k - 1 - o0) % SG_NS) * g.oslot + (go - ost[(k - 1 - o0) % SG_NS]);
            const float* op = ZO ? so : so + ((k + 1 - o0) % SG_NS) * g.oslot + (go - ost[(k + 1 - o0) % SG_NS]);
            const float* bo = sb + ((k - kA) % SG_NB) * g.bslot + ((unsigned)c * L.H + q0 + (unsigned)lane - bst[(k - kA) % SG_NB]);
            float* uo = (RESID ? r : u) + (size_t)c * L.H + q0 + lane;
            const float* uc = u + (size_t)c * L.H + q0 + lane;   // the colour's own values (RESID)
            const float cmz = L.ax[2].cm[k], cpz = L.ax[2].cp[k], dgz = L.ax[2].dg[k];
            const float* cmx = sx + (i1 - 1) * 3 * g.hx1 + lane;
            const float* cpx = cmx + g.hx1;
            const float* dgx = cpx + g.hx1;
#pragma unroll
            for (int v = 0; v < V; v++) {
                if (32 * v < left) {
                    float t = 0.0f;   // ZO: the sum of the six terms over zero neighbours, +0
                    if constexpr (!ZO) {
                        t = cmx[32 * v] * ok[dxm + 32 * v];
                        t = fmaf(cpx[32 * v], ok[dxp + 32 * v], t);
                        t = fmaf(cmy, ok[dym + 32 * v], t);
                        t = fmaf(cpy, ok[dyp + 32 * v], t);
                        t = fmaf(cmz, om[dzm + 32 * v], t);
                        t = fmaf(cpz, op[dzp + 32 * v], t);
                    }
                    if constexpr (RESID) {
                        uo[32 * v] = bo[32 * v] - fmaf(-(dgx[32 * v] + dgy + dgz), __ldg(uc + 32 * v), t);
                    } else {
                        const float acc = bo[32 * v] - t;
                        uo[32 * v] = rb_point32(acc, dgx[32 * v] + dgy + dgz);
                    }
                }
            }
        }
        // every warp is done with plane k - 1 and right-hand side k before their slots refill
        if (__syncthreads_or(bad ? 1 : 0)) {
            failed = true;
            break;
        }
        if (tid == 0) {
            if (!ZO && o_next <= oLast) {   // into plane k - 1's slot
                unsigned st, ln;
                sg_orange(L, c, o_next, j0, nr, st, ln);
                const int q = (o_next - o0) % SG_NS;
                ost[q] = st;
                sg_issue(u, st, ln, so + q * g.oslot, sg_smem(&bar_o[q]));
                o_next++;
            }
            if (b_next <= kB) {      // into right-hand side k's slot
                unsigned st, ln;
                sg_brange(L, c, b_next, j0, nr, st, ln);
                const int q = (b_next - kA) % SG_NB;
                bst[q] = st;
                sg_issue(b, st, ln, sb + q * g.bslot, sg_smem(&bar_b[q]));
                if (RESID) sg_prefetch(u, st, ln);
                b_next++;
            }
        }
    }
    if (tid == 0) {
        // copies issued and not yet waited for land before the block leaves (on the normal path
        // every issued plane has been waited for; after a timeout these waits are bounded too)
        if (failed) {
            for (int p = max(o0, o_next - SG_NS); p < o_next; p++) sg_wait(sg_smem(&bar_o[(p - o0) % SG_NS]), (uint32_t)(((p - o0) / SG_NS) & 1));
            for (int p = max(kA, b_next - SG_NB); p < b_next; p++) sg_wait(sg_smem(&bar_b[(p - kA) % SG_NB]), (uint32_t)(((p - kA) / SG_NB) & 1));
            if (status) atomicMax(status, (int)LASTO_ERR_TIMEOUT);
        }
    }
}

size_t stage_smem(const StageGeom& g)
{
    return sizeof(float) * ((size_t)SG_NS * g.oslot + (size_t)SG_NB * g.bslot + 6 * (size_t)g.hx1);
}

constexpr size_t SG_SMEM_MAX = 200 * 1024;

// the shared-memory opt-in of one instantiation on the current device (done once per device;
// init_stage_attributes does it for all before any graph capture)
template <int V, int MODE>
cudaError_t stage_attr(int dev)
{
    static bool done[64] = {false};
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done[dev]) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k_rbgs_split_stage<V, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)SG_SMEM_MAX);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

template <int V, int MODE>
cudaError_t launch_stage_v(const LevelT<float>& L, float* u, const float* b, int colour, int* status, float* r,
                           cudaStream_t s)
{
    StageGeom g;
    g.tiles_j = (L.ny - 2 + SG_R - 1) / SG_R;
    g.oslot = ((unsigned)(((SG_R + 2) * L.nx + 1) / 2) + 8u + 3u) & ~3u;
    g.bslot = ((unsigned)((SG_R * L.nx + 1) / 2) + 8u + 3u) & ~3u;
    g.hx1 = ((L.nx - 1) / 2 + 3) & ~3;
    const size_t smem = stage_smem(g);
    if (smem > SG_SMEM_MAX) return cudaErrorInvalidValue;
    // one wave: as many plane chunks per tile column as the resident blocks allow
    static int per_sm_cache[64][2] = {{0, 0}};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int per_sm = 0, sms = 0;
    if (per_sm_cache[dev][1] == (int)smem) {
        per_sm = per_sm_cache[dev][0];
    } else {
        e = stage_attr<V, MODE>(dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rbgs_split_stage<V, MODE>, SG_NT, smem);
        if (e != cudaSuccess) return e;
        per_sm_cache[dev][0] = per_sm;
        per_sm_cache[dev][1] = (int)smem;
    }
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int planes = L.nz - 2;
    const int chunks0 = std::max(1, std::min(planes, std::max(1, per_sm) * sms / g.tiles_j));
    g.chunk = (planes + chunks0 - 1) / chunks0;
    const int chunks = (planes + g.chunk - 1) / g.chunk;
    k_rbgs_split_stage<V, MODE><<<(unsigned)(g.tiles_j * chunks), SG_NT, smem, s>>>(L, u, b, colour, g, status, r);
    return cudaGetLastError();
}

}  // namespace

// the grids the staged kernel takes: at least 9 nodes per axis, rows of at most 513 nodes
bool split_stage_ok(int nx, int ny, int nz) { return nx >= 9 && ny >= 9 && nz >= 9 && nx <= 513; }

template <int MODE>
static cudaError_t launch_stage(const LevelT<float>& L, float* u, const float* b, int colour, int* status, float* r,
                                cudaStream_t s)
{
    if (!L.lsh || !split_stage_ok(L.nx, L.ny, L.nz)) return cudaErrorInvalidValue;
    if (((uintptr_t)u & 15u) || ((uintptr_t)b & 15u)) return cudaErrorInvalidValue;
    switch ((L.nx - 1) / 2 <= 256 ? ((L.nx - 1) / 2 + 31) / 32 : 0) {
        case 1: return launch_stage_v<1, MODE>(L, u, b, colour, status, r, s);
        case 2: return launch_stage_v<2, MODE>(L, u, b, colour, status, r, s);
        case 3: return launch_stage_v<3, MODE>(L, u, b, colour, status, r, s);
        case 4: return launch_stage_v<4, MODE>(L, u, b, colour, status, r, s);
        case 5: return launch_stage_v<5, MODE>(L, u, b, colour, status, r, s);
        case 6: return launch_stage_v<6, MODE>(L, u, b, colour, status, r, s);
        case 7: return launch_stage_v<7, MODE>(L, u, b, colour, status, r, s);
        case 8: return launch_stage_v<8, MODE>(L, u, b, colour, status, r, s);
        default: return cudaErrorInvalidValue;
    }
}

// Colour-split FP32 half sweep with staged planes: a grid split_stage_ok accepts, u and b
// 16-byte aligned (else cudaErrorInvalidValue).
cudaError_t launch_split_stage(const LevelT<float>& L, float* u, const float* b, int colour, int* status, cudaStream_t s)
{
    return launch_stage<0>(L, u, b, colour, status, nullptr, s);
}

// The residuals b - A u of the red nodes into r (colour-split storage, red half), staged the
// same way (u, b and r as for launch_split_stage).
cudaError_t launch_split_stage_resid(const LevelT<float>& L, const float* u, const float* b, float* r, int* status,
                                     cudaStream_t s)
{
    if ((uintptr_t)r & 15u) return cudaErrorInvalidValue;
    return launch_stage<1>(L, const_cast<float*>(u), b, 0, status, r, s);
}

// The red half sweep from a black colour that is zero (the first half sweep from u = 0; the
// faces of u zero): neither reads nor stages the black nodes, bitwise the red half sweep over
// zeros.  u and b as for launch_split_stage.
cudaError_t launch_split_stage_first_red(const LevelT<float>& L, float* u, const float* b, int* status, cudaStream_t s)
{
    return launch_stage<2>(L, u, b, 0, status, nullptr, s);
}

// ---------------------------------------------------------------- staged prolongation
// u += P ec on a colour-split fine level (the coarse level natural): the trilinear prolongation
// of Section 3 with the coarse rows a tile reads staged in shared memory.  A block owns 8
// interior fine rows (a warp each, both colours) and a chunk of fine planes; fine plane k reads
// coarse planes k/2 and, for odd k, k/2 + 1 -- rows j0/2 .. (j0 + 7)/2 + 1 of each, one
// contiguous run -- kept in a ring of PS_NS slots with the next plane in flight (a coarse plane
// serves two fine planes).  The fine values are read and written in place, the next fine
// plane's rows brought into L2 by a bulk prefetch one plane ahead.  The node expression is
// k_prolong_add's, so the two are bitwise equal.  ec must be readable up to the next multiple
// of 4 floats past its end (the solver's arrays are padded to 256 bytes).
namespace {

constexpr int PS_R = 8;
constexpr int PS_NT = 32 * PS_R;
constexpr int PS_NS = 3;

struct ProlongGeom {
    int tiles_j, chunk;
    unsigned cslot;   // floats per coarse run slot (a multiple of 4)
    int hx1;          // fine x weights per parity (a multiple of 4)
};

// coarse run of coarse plane K for the tile's fine rows j0 .. j0 + nr - 1
__device__ __forceinline__ void ps_range(const LevelT<float>& C, int K, int j0, int nr, unsigned& st, unsigned& len)
{
    const int Ja = j0 >> 1, Jb = min((j0 + nr - 1) / 2 + 1, C.ny - 1);
    const unsigned lo = ((unsigned)K * (unsigned)C.ny + (unsigned)Ja) * (unsigned)C.nx;
    const unsigned hi = ((unsigned)K * (unsigned)C.ny + (unsigned)Jb + 1u) * (unsigned)C.nx;   // exclusive
    st = lo & ~3u;
    len = ((hi + 3u) & ~3u) - st;
}

template <int V>
__global__ void __launch_bounds__(PS_NT) k_prolong_stage(LevelT<float> F, LevelT<float> C, const float* __restrict__ ec,
                                                         float* __restrict__ u, ProlongGeom g, int* __restrict__ status)
{
    extern __shared__ __align__(16) float sg[];
    __shared__ __align__(8) uint64_t bar[PS_NS];
    __shared__ unsigned cst[PS_NS];
    float* sc = sg;                          // [PS_NS][cslot]
    float* sw = sg + PS_NS * g.cslot;        // fine x weights [2 parities][pl, pr][hx1]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tj = (int)(blockIdx.x % (unsigned)g.tiles_j), kc = (int)(blockIdx.x / (unsigned)g.tiles_j);
    const int j0 = 1 + tj * PS_R;
    const int nr = min(PS_R, F.ny - 1 - j0);
    const int kA = 1 + kc * g.chunk, kB = min(F.nz - 2, kA + g.chunk - 1);
    if (nr <= 0 || kA > kB) return;
    const int nx = F.nx;
    const unsigned nxy = (unsigned)nx * (unsigned)F.ny;
    const int K0 = kA >> 1, KL = (kB >> 1) + 1;   // coarse planes K0 .. KL, in order
    int k_next = K0;
    auto issue = [&](int K) {   // thread 0
        const int q = (K - K0) % PS_NS;
        unsigned st, ln;
        ps_range(C, K, j0, nr, st, ln);
        cst[q] = st;
        const uint32_t b = sg_smem(&bar[q]);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(ln * 4u) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                         sg_smem(sc + q * g.cslot)),
                     "l"(ec + st), "r"(ln * 4u), "r"(b)
                     : "memory");
    };
    auto fine_prefetch = [&](int k) {   // thread 0: plane k's tile rows, both colours, into L2
        for (int t = 0; t < 2; t++) {
            const unsigned lo = (unsigned)t * F.H + (((unsigned)k * nxy + (unsigned)j0 * (unsigned)nx) >> 1);
            const unsigned hi = (unsigned)t * F.H + (((unsigned)k * nxy + (unsigned)(j0 + nr) * (unsigned)nx) >> 1) + 1u;
            sg_prefetch(u, lo & ~3u, (((hi + 3u) & ~3u) - (lo & ~3u)));
        }
    };
    if (tid == 0) {
        for (int q = 0; q < PS_NS; q++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sg_smem(&bar[q])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int t = tid; t < 2 * g.hx1; t += PS_NT) {
        const int par = t / g.hx1, si = t - par * g.hx1;
        const int i = 1 + par + 2 * si;
        const bool in = i < nx - 1;
        sw[(par * 2 + 0) * g.hx1 + si] = in ? F.ax[0].pl[i] : 0.0f;
        sw[(par * 2 + 1) * g.hx1 + si] = in ? F.ax[0].pr[i] : 0.0f;
    }
    __syncthreads();
    if (tid == 0) {
        for (; k_next <= KL && k_next < K0 + PS_NS; k_next++) issue(k_next);
        fine_prefetch(kA);
    }
    const int j = j0 + warp;
    const bool has_row = warp < nr;
    const int nj = (j & 1) ? 2 : 1;
    const float wy0 = has_row ? F.ax[1].pl[j] : 0.0f, wy1 = has_row ? F.ax[1].pr[j] : 0.0f;
    bool failed = false;
    int waited = K0 - 1;   // coarse planes waited for so far
    for (int k = kA; k <= kB; k++) {
        const int K = k >> 1, nk = (k & 1) ? 2 : 1;
        bool bad = false;
        for (int Kw = waited + 1; Kw <= K + nk - 1; Kw++) {
            const int d = Kw - K0;
            if (!bad && !sg_wait(sg_smem(&bar[d % PS_NS]), (uint32_t)((d / PS_NS) & 1))) bad = true;
        }
        waited = max(waited, K + nk - 1);
        if (tid == 0 && k < kB) fine_prefetch(k + 1);
        if (!bad && has_row) {
            const float wz0 = F.ax[2].pl[k], wz1 = F.ax[2].pr[k];
            const float wz[2] = {wz0, wz1}, wy[2] = {wy0, wy1};
            // the coarse row (K, j / 2) of each needed coarse plane, in its slot
            const float* crow[2];
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const int Kc = min(K + c, KL);
                const int q = (Kc - K0) % PS_NS;
                crow[c] = sc + q * g.cslot + ((((unsigned)Kc * (unsigned)C.ny + (unsigned)(j >> 1)) * (unsigned)C.nx) - cst[q]);
            }
#pragma unroll
            for (int t = 0; t < 2; t++) {   // the row's red nodes, then its black ones
                const int i1 = ((t + j + k) & 1) ? 1 : 2;
                const int left = ((nx - i1) >> 1) - lane;
                const int ni = (i1 & 1) ? 2 : 1;   // the parity of i is the run's
                float* ur = u + (size_t)t * F.H + ((((unsigned)k * nxy + (unsigned)j * (unsigned)nx + (unsigned)i1) >> 1) + lane);
                const float* wx0 = sw + (i1 - 1) * 2 * g.hx1 + lane;
                const float* wx1 = wx0 + g.hx1;
                float uv[V];
#pragma unroll
                for (int v = 0; v < V; v++) uv[v] = 32 * v < left ? ur[32 * v] : 0.0f;
#pragma unroll
                for (int v = 0; v < V; v++) {
                    if (32 * v >= left) continue;
                    const int i = i1 + 2 * (lane + 32 * v);
                    const float wx[2] = {wx0[32 * v], wx1[32 * v]};
                    float e = 0.0f;
#pragma unroll
                    for (int c = 0; c < 2; c++)
#pragma unroll
                        for (int bb = 0; bb < 2; bb++) {
                            if (c >= nk || bb >= nj) continue;
                            const float* r = crow[c] + bb * C.nx + (i >> 1);
                            const float sv = (ni == 2) ? fmaf(wx[0], r[0], wx[1] * r[1]) : r[0];
                            e = fmaf(wz[c] * wy[bb], sv, e);
                        }
                    ur[32 * v] = uv[v] + e;
                }
            }
        }
        if (__syncthreads_or(bad ? 1 : 0)) {
            failed = true;
            break;
        }
        // after an odd fine plane its lower coarse plane is done: its slot takes the next one
        if (tid == 0 && (k & 1) && k_next <= KL) issue(k_next++);
    }
    if (tid == 0 && failed) {
        for (int K = max(K0, k_next - PS_NS); K < k_next; K++)
            sg_wait(sg_smem(&bar[(K - K0) % PS_NS]), (uint32_t)(((K - K0) / PS_NS) & 1));
        if (status) atomicMax(status, (int)LASTO_ERR_TIMEOUT);
    }
}

template <int V>
cudaError_t launch_prolong_stage_v(const LevelT<float>& F, const LevelT<float>& C, const float* ec, float* u,
                                   int* status, cudaStream_t s)
{
    static bool attr[64] = {false};
    static int per_sm_cache[64][2] = {{0, 0}};
    ProlongGeom g;
    g.tiles_j = (F.ny - 2 + PS_R - 1) / PS_R;
    g.cslot = (((unsigned)(PS_R / 2 + 2) * (unsigned)C.nx) + 8u + 3u) & ~3u;
    g.hx1 = ((F.nx - 1) / 2 + 3) & ~3;
    const size_t smem = sizeof(float) * ((size_t)PS_NS * g.cslot + 4 * (size_t)g.hx1);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        e = cudaFuncSetAttribute(k_prolong_stage<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    int per_sm = 0, sms = 0;
    if (per_sm_cache[dev][1] == (int)smem) {
        per_sm = per_sm_cache[dev][0];
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prolong_stage<V>, PS_NT, smem);
        if (e != cudaSuccess) return e;
        per_sm_cache[dev][0] = per_sm;
        per_sm_cache[dev][1] = (int)smem;
    }
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // chunks of an even number of fine planes (a coarse plane serves a pair)
    const int planes = F.nz - 2;
    const int chunks0 = std::max(1, std::min(planes, std::max(1, per_sm) * sms / g.tiles_j));
    g.chunk = (planes + chunks0 - 1) / chunks0;
    g.chunk += g.chunk & 1;
    const int chunks = (planes + g.chunk - 1) / g.chunk;
    k_prolong_stage<V><<<(unsigned)(g.tiles_j * chunks), PS_NT, smem, s>>>(F, C, ec, u, g, status);
    return cudaGetLastError();
}

}  // namespace

// u += P ec, fine level colour-split (a grid split_stage_ok accepts, u 16-byte aligned), coarse
// level natural with every axis (n + 1) / 2 of the fine one; ec readable to the next multiple of
// 4 floats past its end
cudaError_t launch_prolong_stage(const LevelT<float>& F, const LevelT<float>& C, const float* ec, float* u, int* status,
                                 cudaStream_t s)
{
    if (!F.lsh || C.lsh || !split_stage_ok(F.nx, F.ny, F.nz) || ((uintptr_t)u & 15u) || ((uintptr_t)ec & 15u))
        return cudaErrorInvalidValue;
    if (C.nx != (F.nx + 1) / 2 || C.ny != (F.ny + 1) / 2 || C.nz != (F.nz + 1) / 2) return cudaErrorInvalidValue;
    switch ((F.nx - 1) / 2 <= 256 ? ((F.nx - 1) / 2 + 31) / 32 : 0) {
        case 1: return launch_prolong_stage_v<1>(F, C, ec, u, status, s);
        case 2: return launch_prolong_stage_v<2>(F, C, ec, u, status, s);
        case 3: return launch_prolong_stage_v<3>(F, C, ec, u, status, s);
        case 4: return launch_prolong_stage_v<4>(F, C, ec, u, status, s);
        case 5: return launch_prolong_stage_v<5>(F, C, ec, u, status, s);
        case 6: return launch_prolong_stage_v<6>(F, C, ec, u, status, s);
        case 7: return launch_prolong_stage_v<7>(F, C, ec, u, status, s);
        case 8: return launch_prolong_stage_v<8>(F, C, ec, u, status, s);
        default: return cudaErrorInvalidValue;
    }
}

void init_stage_attributes()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    stage_attr<1, 0>(dev), stage_attr<2, 0>(dev), stage_attr<3, 0>(dev), stage_attr<4, 0>(dev);
    stage_attr<5, 0>(dev), stage_attr<6, 0>(dev), stage_attr<7, 0>(dev), stage_attr<8, 0>(dev);
    stage_attr<1, 1>(dev), stage_attr<2, 1>(dev), stage_attr<3, 1>(dev), stage_attr<4, 1>(dev);
    stage_attr<5, 1>(dev), stage_attr<6, 1>(dev), stage_attr<7, 1>(dev), stage_attr<8, 1>(dev);
    stage_attr<1, 2>(dev), stage_attr<2, 2>(dev), stage_attr<3, 2>(dev), stage_attr<4, 2>(dev);
    stage_attr<5, 2>(dev), stage_attr<6, 2>(dev), stage_attr<7, 2>(dev), stage_attr<8, 2>(dev);
}

}  // namespace lasto
