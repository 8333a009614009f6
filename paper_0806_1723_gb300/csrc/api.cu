// C ABI of the GB300 LASTO interstitial Poisson step: handle, workspace, CUDA-graph
// plan of one solve, and the single-operation entry points.
//
// One solve is captured once into a CUDA graph and replayed: setup (mesh tables,
// coarse eigenvectors, sphere parameters), deposit, multipoles, faces, then a
// conditional WHILE node whose body is one multigrid-preconditioned CG iteration (or
// one V-cycle), and whose condition is set on the device by the convergence test, so
// the iteration runs with no host round trip.  Then the true residual, the projection
// and the stats.
#include <algorithm>
#include <cstring>
#include <cstdio>
#include <map>
#include <array>
#include <algorithm>
#include <new>
#include <vector>

#include "ctl.cuh"
#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

using namespace lasto;

namespace {

struct Scratch {
    void* p = nullptr;
    cudaStream_t s;
    explicit Scratch(size_t bytes, cudaStream_t st) : s(st)
    {
        if (bytes && cudaMallocAsync(&p, bytes, s) != cudaSuccess) p = nullptr;
    }
    ~Scratch()
    {
        if (p) cudaFreeAsync(p, s);
    }
    template <typename T>
    T* as() const { return reinterpret_cast<T*>(p); }
};

// A bump allocator over one device pool (all pieces 256-byte aligned).
struct Carver {
    char* base;
    size_t cap, off = 0;
    bool ok = true;
    template <typename T>
    T* take(size_t count)
    {
        const size_t bytes = ((count * sizeof(T)) + 255) & ~size_t(255);
        if (off + bytes > cap) {
            ok = false;
            return nullptr;
        }
        T* p = reinterpret_cast<T*>(base + off);
        off += bytes;
        return p;
    }
};

// How one level is smoothed: in-place half sweeps (block size nt) or fused passes ping-ponging
// with a partner array: fused = 1, the z-slab / register-column kernels (shape sh); fused = 2,
// the FP32 wavefront sweep over bulk-copied row chunks (sh.tx columns, sh.ty rows); fused = 3,
// in-place half sweeps over colour-split storage (FP32, block size nt), which the finest level
// of a cluster then uses for all its FP32 arrays (another level with these dimensions runs the
// natural in-place sweeps with the same block size).
struct SmoothChoice {
    int fused = 0;
    int nt = 256;
    SlabShape sh{0, 0, 0, 0};
    float us = 0.0f;   // measured time of one pre-smoothing phase
};

// Everything one cluster's solve touches on the device.
struct ClusterPlan {
    int L = 0;
    LevelStore lv[MAX_LEVELS];
    double *p = nullptr, *q = nullptr, *z = nullptr;  // level-0 CG vectors (FP64)
    float *e32 = nullptr, *p32 = nullptr, *q32 = nullptr;  // level-0 inner CG vectors (FP32)
    double* rec = nullptr;                            // sphere records
    double* mom = nullptr;                            // multipole scratch
    double* part = nullptr;                           // reduction partials
    int nparts = 0;
    double* Q = nullptr;
    Ctl* ctl = nullptr;
    CoarseEig* eig = nullptr;
    int* status = nullptr;              // [0] status, [1] reduction ticket counter
    lasto_stats* stats_dev = nullptr;
    // learned guess: the 33^3 subgrid (every gm-th node) and the level gl it is resampled from
    double *gax[3] = {nullptr, nullptr, nullptr};
    double *bG = nullptr, *fG = nullptr, *uG = nullptr;
    int gm[3] = {0, 0, 0};
    int gl = -1;      // -1: no learned guess for this cluster
    int gslot = -1;   // its grid in the network's batch
    const lasto_raw_cluster* raw = nullptr;   // raw-density input (null: the synthetic model)
    Red red(int op, cudaGraphConditionalHandle cond = 0, int use_cond = 0) const
    {
        return Red{part, reinterpret_cast<unsigned int*>(status + 1), ctl, op, cond, use_cond};
    }
};

size_t cluster_bytes(const int n[3], int n_atoms)
{
    // generous upper bound computed by a dry run of the carver
    Carver c{nullptr, ~size_t(0) >> 1};
    int nn[3] = {n[0], n[1], n[2]};
    const int L = num_levels(nn);
    if (L < 1) return 0;
    for (int l = 0; l < L; l++) {
        const size_t N = (size_t)nn[0] * nn[1] * nn[2];
        for (int d = 0; d < 3; d++) c.take<double>(axis_pool_doubles(nn[d]));
        c.take<double>(N);          // inv_diag
        for (int t = 0; t < 4; t++) c.take<double>(N);
        for (int t = 0; t < 3; t++) c.take<float>(N);
        if (l == 0) {
            for (int t = 0; t < 3; t++) c.take<double>(N);
            for (int t = 0; t < 3; t++) c.take<float>(N);
        }
        for (int d = 0; d < 3; d++) nn[d] = (nn[d] + 1) / 2;
    }
    c.take<double>((size_t)SPHERE_REC_DOUBLES * std::max(n_atoms, 1));
    c.take<double>(multipole_scratch_doubles(n));
    c.take<double>(((size_t)n[0] * n[1] * n[2] + 255) / 256 + 64);
    c.take<double>(32);
    c.take<Ctl>(1);
    c.take<CoarseEig>(1);
    c.take<int>(4);
    c.take<lasto_stats>(1);
    for (int d = 0; d < 3; d++) c.take<double>(GUESS_N);
    for (int t = 0; t < 3; t++) c.take<double>((size_t)GUESS_N * GUESS_N * GUESS_N);
    return c.off;
}

bool carve_cluster(Carver& c, const int n[3], int n_atoms, ClusterPlan& P)
{
    int nn[3] = {n[0], n[1], n[2]};
    P.L = num_levels(nn);
    if (P.L < 1) return false;
    for (int l = 0; l < P.L; l++) {
        LevelStore& S = P.lv[l];
        const size_t N = (size_t)nn[0] * nn[1] * nn[2];
        for (int d = 0; d < 3; d++) {
            S.n[d] = nn[d];
            double* pool = c.take<double>(axis_pool_doubles(nn[d]));
            if (!pool) return false;
            carve_axis(&S.ax[d], nn[d], pool);
        }
        S.inv_diag = c.take<double>(N);
        S.u = c.take<double>(N);
        S.b = c.take<double>(N);
        S.r = c.take<double>(N);
        S.u2 = c.take<double>(N);
        S.u32 = c.take<float>(N);
        S.b32 = c.take<float>(N);
        S.r32 = c.take<float>(N);
        if (l == 0) {
            P.p = c.take<double>(N);
            P.q = c.take<double>(N);
            P.z = c.take<double>(N);
            P.e32 = c.take<float>(N);
            P.p32 = c.take<float>(N);
            P.q32 = c.take<float>(N);
        }
        for (int d = 0; d < 3; d++) nn[d] = (nn[d] + 1) / 2;
    }
    P.rec = c.take<double>((size_t)SPHERE_REC_DOUBLES * std::max(n_atoms, 1));
    P.mom = c.take<double>(multipole_scratch_doubles(n));
    P.nparts = (int)(((size_t)n[0] * n[1] * n[2] + 255) / 256);
    P.part = c.take<double>((size_t)P.nparts + 64);
    P.Q = c.take<double>(32);
    P.ctl = c.take<Ctl>(1);
    P.eig = c.take<CoarseEig>(1);
    P.status = c.take<int>(4);
    P.stats_dev = c.take<lasto_stats>(1);
    for (int d = 0; d < 3; d++) P.gax[d] = c.take<double>(GUESS_N);
    P.bG = c.take<double>((size_t)GUESS_N * GUESS_N * GUESS_N);
    P.fG = c.take<double>((size_t)GUESS_N * GUESS_N * GUESS_N);
    P.uG = c.take<double>((size_t)GUESS_N * GUESS_N * GUESS_N);
    return c.ok;
}

bool valid_n(const int n[3])
{
    for (int d = 0; d < 3; d++)
        if (n[d] < 3 || n[d] % 2 == 0) return false;
    if ((size_t)n[0] * n[1] * n[2] >= (size_t(1) << 31)) return false;   // kernels index with 31 bits
    int nn[3] = {n[0], n[1], n[2]};
    return num_levels(nn) >= 1;
}

// one block per interior (j, k) row, the row's interior nodes four per thread (loads first)
__global__ void __launch_bounds__(128) k_copy_interior(const double* __restrict__ src, double* __restrict__ dst, int nx,
                                                       int ny, int nz)
{
    const int my = ny - 2;
    const int row = (int)blockIdx.x;
    const int k = row / my + 1, j = row - (k - 1) * my + 1;
    const size_t base = ((size_t)k * ny + j) * nx;
    for (int i0 = 1 + (int)threadIdx.x; i0 < nx - 1; i0 += 4 * 128) {
        double v[4];
#pragma unroll
        for (int q = 0; q < 4; q++) v[q] = i0 + 128 * q < nx - 1 ? src[base + i0 + 128 * q] : 0.0;
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (i0 + 128 * q < nx - 1) dst[base + i0 + 128 * q] = v[q];
    }
}

// true_is_last: the loop's last residual is already the true FP64 residual of the final iterate
// (defect correction: each step ends with it, and the iterate does not change after it)
__global__ void k_write_stats(const Ctl* __restrict__ ctl, const int* __restrict__ status, int guess,
                              int true_is_last, lasto_stats* out)
{
    lasto_stats s;
    s.guess = guess;
    s.cycles = ctl->iter;
    s.rel_resid = true_is_last ? ctl->rel : ctl->true_rel;
    s.bnorm = ctl->bnorm;
    s.status = status[0] != 0 ? status[0] : ctl->status;
    s.outer = ctl->outer;
    *out = s;
}

}  // namespace

struct lasto_poisson {
    lasto_config cfg;
    Err err;
    int device = 0;
    char* pool = nullptr;
    size_t pool_bytes = 0;
    double* quad = nullptr;
    int nq = 0;
    cudaStream_t cs = nullptr, cs2 = nullptr, cs3 = nullptr;
    cudaEvent_t ev_origin = nullptr;
    // per batch slot: the cluster's branch stream, its setup stream and fork/join/done events
    std::vector<cudaStream_t> bs, ss;
    std::vector<cudaEvent_t> ef, ej, ed;
    std::vector<cudaEvent_t> es, eb;     // per slot: iteration prologue done; lockstep loops done
    // lockstep batches (launch = 2): the members' kernel arguments, on the device
    char* bat_args = nullptr;
    size_t bat_bytes = 0;
    // cached graph
    std::vector<char> key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int n_clusters = 0;
    std::vector<ClusterPlan> plans;
    lasto_stats* stats_pinned = nullptr;
    int kernels_fixed = -1, kernels_iter = -1, kernels_outer = 0;
    std::vector<cudaGraph_t> bodies, outer_bodies;
    // smoother choice per level shape {nx, ny, nz, element bytes}: measured once, reused
    std::map<std::array<int, 4>, SmoothChoice> tune;
    GuessNet* net = nullptr;             // learned initial guess (optional)
    std::vector<lasto_raw_cluster> raw_copy;   // raw-density inputs of the current solve call
    std::vector<cudaEvent_t> eg;         // per slot: features written
    cudaEvent_t ev_net = nullptr;        // network forward done
    // the last solve's work on the caller's stream (graph launch and stats copy): waited for
    // before the workspace is re-carved, the graph replaced, or the handle freed
    cudaEvent_t ev_launch = nullptr;
};

namespace {

// A named range on the host thread's NVTX timeline (shown by profilers beside the kernels it
// enqueues; a no-op without a profiler attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

int fail(lasto_poisson* h, int code, const std::string& msg)
{
    if (h) {
        h->err.code = code;
        h->err.msg = msg;
    }
    return code;
}

#define TRY(call)                                                            \
    do {                                                                     \
        cudaError_t c_ = (call);                                             \
        if (c_ != cudaSuccess) return set_cuda_error(&h->err, c_, #call);    \
    } while (0)

// ---------------------------------------------------------------- cycles (enqueue only)
template <typename T>
struct Arr;
template <>
struct Arr<double> {
    static double* partner(LevelStore& s) { return s.u2; }
    static double* u(LevelStore& s) { return s.u; }
    static double* b(LevelStore& s) { return s.b; }
    static double* r(LevelStore& s) { return s.r; }
    static LevelT<double> view(const LevelStore& s) { return s.view64(); }
};
template <>
struct Arr<float> {
    static float* partner(LevelStore& s) { return s.r32; }   // r32 is free in the FP32 cycle
    static float* u(LevelStore& s) { return s.u32; }
    static float* b(LevelStore& s) { return s.b32; }
    static float* r(LevelStore& s) { return s.r32; }
    static LevelT<float> view(const LevelStore& s) { return s.view32(); }
};

// ---------------------------------------------------------------- smoothing and its tuner
// `nu` red-black sweeps starting with colour `first`.  In place, or as fused passes from
// `cur` into the other of {home, partner}; cur follows the data.
template <typename T>
cudaError_t smooth(const LevelT<T>& V, T*& cur, T* partner, T* home, const T* b, int nu, int first,
                   const SmoothChoice& ch, int* status, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (ch.fused == 2) {
        if constexpr (sizeof(T) == 4) {
            for (int m = 0; m < nu && e == cudaSuccess; m++) {
                T* dst = cur == home ? partner : home;
                e = launch_rb_wave(V, cur, dst, b, first, ch.sh, s);
                cur = dst;
            }
            return e;
        }
        return cudaErrorInvalidValue;
    }
    if (ch.fused == 0 || ch.fused == 3) {   // the view's storage order picks the kernel
        for (int it = 0; it < nu && e == cudaSuccess; it++) {
            e = launch_rbgs<T>(V, cur, b, first, s, ch.nt, status);
            if (e == cudaSuccess) e = launch_rbgs<T>(V, cur, b, 1 - first, s, ch.nt, status);
        }
        return e;
    }
    const int ns = ch.sh.ns, full = nu / ns, rest = nu % ns;
    for (int m = 0; m < full + (rest ? 1 : 0) && e == cudaSuccess; m++) {
        SlabShape sh = ch.sh;
        if (m == full) {
            sh = slab_default_shape(rest, sizeof(T));
            sh.kz = ch.sh.kz;
        }
        T* dst = cur == home ? partner : home;
        e = launch_rb_slab<T>(V, cur, dst, b, first, 0, sh, s);
        cur = dst;
    }
    return e;
}

int fused_passes(int nu, int ns) { return nu / ns + (nu % ns ? 1 : 0); }

bool choice_usable(const lasto_poisson* h, const SmoothChoice& c, size_t elem)
{
    if (c.fused == 3 && c.nt == RBGS_STAGED) return elem == 4;
    if (c.fused == 0 || c.fused == 3)
        return (c.fused == 0 || elem == 4) && (c.nt == 0 || (c.nt >= 32 && c.nt <= 512 && c.nt % 32 == 0));
    if (c.fused == 2) return elem == 4 && wave_shape_ok(c.sh) && (h->cfg.nu1 + h->cfg.nu2) % 2 == 0;
    // the pre- and post-smoothing passes together must return the data to its home array
    return slab_shape_ok(c.sh, elem) && (fused_passes(h->cfg.nu1, c.sh.ns) + fused_passes(h->cfg.nu2, c.sh.ns)) % 2 == 0;
}

template <typename T>
SmoothChoice smooth_choice(const lasto_poisson* h, const LevelStore& S)
{
    auto it = h->tune.find({S.n[0], S.n[1], S.n[2], (int)sizeof(T)});
    if (it != h->tune.end() && choice_usable(h, it->second, sizeof(T))) return it->second;
    return SmoothChoice{};
}

// Time the candidates on this level's own arrays (zeroed; the stream is idle and not being
// captured) and keep the fastest pre-smoothing phase.
template <typename T>
int tune_level(lasto_poisson* h, LevelStore& S, bool finest, cudaStream_t st)
{
    const std::array<int, 4> key{S.n[0], S.n[1], S.n[2], (int)sizeof(T)};
    if (h->tune.count(key)) return LASTO_OK;
    LevelT<T> V = Arr<T>::view(S);
    set_split(V, false);
    LevelT<T> Vs = V;   // the same arrays read as colour-split storage
    set_split(Vs, true);
    T* u = Arr<T>::u(S);
    T* partner = Arr<T>::partner(S);
    T* b = Arr<T>::b(S);
    TRY(cudaMemsetAsync(u, 0, sizeof(T) * S.N(), st));
    TRY(cudaMemsetAsync(partner, 0, sizeof(T) * S.N(), st));
    TRY(cudaMemsetAsync(b, 0, sizeof(T) * S.N(), st));
    std::vector<SmoothChoice> cand;
    for (int nt : {128, 256, 512}) {
        SmoothChoice c;
        c.nt = nt;
        cand.push_back(c);
    }
    if ((S.n[0] + 1) / 2 <= 512) {
        SmoothChoice c;
        c.nt = 0;   // one block per row
        cand.push_back(c);
    }
    const bool f32 = sizeof(T) == 4;
    if (f32 && finest)
        for (int nt : {128, 256, 512, 0, RBGS_STAGED}) {
            if (nt == 0 && (S.n[0] + 1) / 2 > 512) continue;
            if (nt == RBGS_STAGED && !split_stage_ok(S.n[0], S.n[1], S.n[2])) continue;
            SmoothChoice c;
            c.fused = 3;
            c.nt = nt;
            cand.push_back(c);
        }
    for (int ty : f32 ? std::vector<int>{6, 14} : std::vector<int>{2, 6})
        for (int kz : {16, 32}) {
            SmoothChoice c;
            c.fused = 1;
            c.sh = SlabShape{62, ty, kz, 1};
            cand.push_back(c);
        }
    for (SlabShape sh : {SlabShape{64, 16, 32, 2}, SlabShape{32, 8, 16, 2}}) {
        SmoothChoice c;
        c.fused = 1;
        c.sh = sh;
        cand.push_back(c);
    }
    if (f32 && wave_level_ok(S.n[0], S.n[1], S.n[2]))
        for (int ty : {8, 16})
            for (int tx : {48, 60}) {
                SmoothChoice c;
                c.fused = 2;
                c.sh = SlabShape{tx, ty, 8, 1};
                cand.push_back(c);
            }
    cudaEvent_t e0, e1;
    TRY(cudaEventCreate(&e0));
    TRY(cudaEventCreate(&e1));
    SmoothChoice best;
    best.us = 1e30f;
    for (const SmoothChoice& c : cand) {
        if (!choice_usable(h, c, sizeof(T))) continue;
        T* cur = u;
        const LevelT<T>& Vc = c.fused == 3 ? Vs : V;
        cudaError_t e = smooth<T>(Vc, cur, partner, u, b, h->cfg.nu1, 0, c, nullptr, st);   // warm
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && e == cudaSuccess; r++)
            e = smooth<T>(Vc, cur, partner, u, b, h->cfg.nu1, 0, c, nullptr, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return set_cuda_error(&h->err, e, "smoother tuning");
        }
        const float us = ms * 1000.0f / 3.0f;
        if (us < best.us) {
            best = c;
            best.us = us;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->tune[key] = best;
    return LASTO_OK;
}

// First level run by the one-block bottom kernel (its correction starts at zero, so not
// level 0), or -1 when every level is launched separately.  FP32 only: one SM's FP64 units
// are far too slow for even a 17^3 level, while FP32 work this small is pure launch latency.
int bottom_level(const ClusterPlan& P)
{
    for (int l = 1; l < P.L - 1; l++)
        if (P.lv[l].N() <= BOTTOM_MAX_NODES && P.L - l <= BOTTOM_MAX_LEVELS) return l;
    return -1;
}

template <typename T>
int enqueue_cycle(lasto_poisson* h, ClusterPlan& P, int l, T* u, T* b, T* r, bool fcycle, bool sym, cudaStream_t s,
                  bool zero_start = false)
{
    LevelStore& S = P.lv[l];
    const LevelT<T> V = Arr<T>::view(S);
    const int nu1 = (l == 0 && h->cfg.nu_fine > 0) ? h->cfg.nu_fine : h->cfg.nu1;
    const int nu2 = (l == 0 && h->cfg.nu_fine > 0) ? h->cfg.nu_fine : h->cfg.nu2;
    if (sizeof(T) == 4 && !fcycle && l > 0 && l == bottom_level(P)) {
        BottomArgs<T> a;
        a.nlev = P.L - l;
        for (int q = 0; q < a.nlev; q++) {
            a.lv[q] = Arr<T>::view(P.lv[l + q]);
            a.u[q] = Arr<T>::u(P.lv[l + q]);
            a.b[q] = Arr<T>::b(P.lv[l + q]);
        }
        a.eig = P.eig;
        a.nu1 = h->cfg.nu_coarse;   // one-block levels: their own (symmetric) sweep count
        a.nu2 = h->cfg.nu_coarse;
        a.sym = sym ? 1 : 0;
        TRY(launch_bottom<T>(a, s));
        return LASTO_OK;
    }
    if (l == P.L - 1) {
        if (l == 0) {
            TRY(launch_residual<T>(V, u, b, r, s));
            TRY(launch_coarse_apply<T>(V, P.eig, r, u, true, s));
        } else {
            TRY(launch_coarse_apply<T>(V, P.eig, b, u, false, s));
        }
        return LASTO_OK;
    }
    SmoothChoice ch = smooth_choice<T>(h, S);
    if (V.lsh) {   // colour-split storage: in-place sweeps only
        if (ch.fused != 0 && ch.fused != 3) ch = SmoothChoice{};
        ch.fused = 3;
    } else if (ch.fused == 3) {
        ch.fused = 0;
        if (ch.nt == RBGS_STAGED) ch.nt = 0;   // natural storage: one block per row
    }
    T* cur = u;   // fused passes move the iterate between u and the partner array
    if (zero_start && sizeof(T) == 4 && nu1 >= 1 && (ch.fused == 0 || ch.fused == 3)) {
        // from u = 0 (faces zero) the first red half sweep is a point update
        if constexpr (sizeof(T) == 4) {
            if (V.lsh && ch.nt == RBGS_STAGED)
                TRY(launch_split_stage_first_red(V, u, b, P.status, s));
            else
                TRY(launch_first_red32(V, u, b, s));
        }
        TRY(launch_rbgs<T>(V, u, b, 1, s, ch.nt, P.status));
        TRY(smooth<T>(V, cur, Arr<T>::partner(S), u, b, nu1 - 1, 0, ch, P.status, s));
    } else {
        TRY(smooth<T>(V, cur, Arr<T>::partner(S), u, b, nu1, 0, ch, P.status, s));
    }
    LevelStore& C = P.lv[l + 1];
    const LevelT<T> VC = Arr<T>::view(C);
    if (sizeof(T) == 4) {
        // FP32: form the 27 fine residuals inside the restriction (cheaper than a pass)
        // after nu1 >= 1 sweeps that end on the black half sweep the black residuals are zero
        // (over colour-split storage the red residuals may go through the free r array first)
        TRY(launch_resid_restrict<T>(V, VC, cur, b, Arr<T>::b(C), Arr<T>::u(C), nu1 > 0, s, V.lsh ? r : nullptr,
                                     P.status));
    } else {
        // FP64: each residual once (FP64 arithmetic, not bandwidth, bounds this chip)
        TRY(launch_residual<T>(V, cur, b, r, s));
        TRY(launch_restrict<T>(V, VC, r, Arr<T>::b(C), s));
        TRY(cudaMemsetAsync(Arr<T>::u(C), 0, sizeof(T) * C.N(), s));
    }
    int st = enqueue_cycle<T>(h, P, l + 1, Arr<T>::u(C), Arr<T>::b(C), Arr<T>::r(C), fcycle, sym, s);
    if (st) return st;
    if (fcycle) {
        st = enqueue_cycle<T>(h, P, l + 1, Arr<T>::u(C), Arr<T>::b(C), Arr<T>::r(C), false, sym, s);
        if (st) return st;
    }
    TRY(launch_prolong_add<T>(V, VC, Arr<T>::u(C), cur, s, P.status));
    TRY(smooth<T>(V, cur, Arr<T>::partner(S), u, b, nu2, sym ? 1 : 0, ch, P.status, s));
    if (cur != u) return fail(h, LASTO_ERR_INVALID_ARG, "smoother passes do not return to the level array");
    return LASTO_OK;
}

int enqueue_setup(lasto_poisson* h, ClusterPlan& P, const lasto_cluster& cl, cudaStream_t s)
{
    // the FP64 smoother (plain preconditioner, stationary cycles) reads a stored inverse diagonal
    const bool fp64 = h->cfg.precision == LASTO_PREC_FP64 || h->cfg.cycle != LASTO_CYCLE_PCG;
    for (int l = 0; l < P.L; l++) {
        const double* src[3];
        int stride;
        if (l == 0) {
            src[0] = cl.x;
            src[1] = cl.y;
            src[2] = cl.z;
            stride = 1;
        } else {
            for (int d = 0; d < 3; d++) src[d] = P.lv[l - 1].ax[d].c;
            stride = 2;
        }
        TRY(launch_level_tables(P.lv[l], nullptr, src, stride, s));
        if (fp64 && l < P.L - 1) TRY(launch_inv_diag(P.lv[l], s));
    }
    TRY(launch_coarse_eig(P.lv[P.L - 1], P.eig, s));
    return LASTO_OK;
}

RawArgs raw_args(const lasto_raw_cluster& r)
{
    RawArgs a;
    a.na = r.n_atoms;
    a.pos = r.pos;
    a.Z = r.Z;
    a.R = r.R;
    for (int d = 0; d < 3; d++) a.n[d] = r.n[d];
    a.ax[0] = r.x;
    a.ax[1] = r.y;
    a.ax[2] = r.z;
    a.ne = r.density;
    a.n_rad = r.n_rad;
    a.r_min = r.r_min;
    a.rho00 = r.rho00;
    return a;
}

// the geometry part of a raw cluster as a lasto_cluster (no model arrays)
lasto_cluster cluster_of(const lasto_raw_cluster& r)
{
    lasto_cluster c;
    std::memset(&c, 0, sizeof(c));
    c.n_atoms = r.n_atoms;
    c.pos = r.pos;
    c.Z = r.Z;
    c.R = r.R;
    for (int d = 0; d < 3; d++) {
        c.n[d] = r.n[d];
        c.centre[d] = r.centre[d];
    }
    c.x = r.x;
    c.y = r.y;
    c.z = r.z;
    return c;
}

int enqueue_rhs(lasto_poisson* h, ClusterPlan& P, const lasto_cluster& cl, const double* guess, cudaStream_t s)
{
    LevelStore& F = P.lv[0];
    const int* n = cl.n;
    if (P.raw) {
        const RawArgs ra = raw_args(*P.raw);
        TRY(launch_raw_sphere_params(ra, P.rec, P.status, s));
        TRY(launch_raw_deposit(ra, P.rec, F.b, nullptr, P.status, s));
    } else {
        TRY(launch_sphere_params(cl, cl.x, cl.y, cl.z, P.rec, nullptr, nullptr, nullptr, nullptr, P.status, s));
        TRY(launch_deposit(cl, P.rec, h->cfg.precision, F.b, nullptr, nullptr, nullptr, P.status, s));
    }
    double* tabs = P.mom;
    double* rowm = tabs + 5 * ((size_t)n[0] + n[1] + n[2]);
    double* plane = rowm + 5 * (size_t)n[1] * n[2];
    TRY(cudaMemsetAsync(F.u, 0, sizeof(double) * F.N(), s));
    if (h->cfg.boundary == LASTO_BC_MULTIPOLE) {
        TRY(launch_multipoles(n, cl.x, cl.y, cl.z, F.b, cl.centre, tabs, rowm, plane, P.Q, s));
        TRY(launch_boundary_fill(n, cl.x, cl.y, cl.z, cl.centre[0], cl.centre[1], cl.centre[2], P.Q, F.u, s));
    } else if (h->cfg.boundary == LASTO_BC_EXACT) {
        TRY(launch_boundary_exact(cl, tabs, F.u, s));   // the multipole scratch holds the moments
    }   // LASTO_BC_ZERO: the faces stay 0 (Eq. 3.3)
    if (guess) {
        k_copy_interior<<<(unsigned)((n[1] - 2) * (n[2] - 2)), 128, 0, s>>>(guess, F.u, n[0], n[1], n[2]);
        TRY(cudaGetLastError());
    }
    return LASTO_OK;
}

// Setup and right-hand side of one cluster.  The mesh tables and the coarse eigenvectors
// depend only on the mesh and run on a second stream beside the sphere parameters,
// deposit, multipoles and faces; the two branches join before the iteration.
int enqueue_prologue(lasto_poisson* h, ClusterPlan& P, const lasto_cluster& cl, const double* guess, cudaStream_t s,
                     int slot)
{
    cudaStream_t side = h->ss[slot];
    TRY(cudaEventRecord(h->ef[slot], s));
    TRY(cudaStreamWaitEvent(side, h->ef[slot], 0));
    int st = enqueue_setup(h, P, cl, side);
    if (st) return st;
    TRY(cudaEventRecord(h->ej[slot], side));
    TRY(cudaMemsetAsync(P.status, 0, sizeof(int) * 4, s));
    if ((st = enqueue_rhs(h, P, cl, guess, s))) return st;
    TRY(cudaStreamWaitEvent(s, h->ej[slot], 0));
    return LASTO_OK;
}

// ---------------------------------------------------------------- learned guess stages
// Which clusters get the learned guess: every axis n = 32 m + 1 (the 33^3 subgrid takes every
// m-th node), a network loaded and no caller guess.  gl = the deepest level with at least 33
// nodes per axis (the subgrid itself for 33, 65, 129, 257, ... nodes).
int plan_guesses(lasto_poisson* h, const lasto_cluster* cls, int nc, const double* guess)
{
    int k = 0;
    for (int c = 0; c < nc; c++) {
        ClusterPlan& P = h->plans[c];
        P.gl = -1;
        P.gslot = -1;
        if (!h->net || guess) continue;
        bool ok = true;
        for (int d = 0; d < 3; d++) {
            const int n = cls[c].n[d];
            ok = ok && n >= GUESS_N && (n - 1) % (GUESS_N - 1) == 0;
            P.gm[d] = (n - 1) / (GUESS_N - 1);
        }
        if (!ok || k >= guess_net_capacity(h->net)) continue;
        int gl = 0;
        while (gl + 1 < P.L && P.lv[gl + 1].n[0] >= GUESS_N && P.lv[gl + 1].n[1] >= GUESS_N &&
               P.lv[gl + 1].n[2] >= GUESS_N)
            gl++;
        P.gl = gl;
        P.gslot = k++;
    }
    return k;
}

// network input of one cluster (after its right-hand side and mesh tables)
int enqueue_guess_in(lasto_poisson* h, ClusterPlan& P, const lasto_cluster& cl, cudaStream_t s)
{
    if (P.gl < 0) return LASTO_OK;
    const double* ax[3] = {cl.x, cl.y, cl.z};
    const int G[3] = {GUESS_N, GUESS_N, GUESS_N};
    for (int d = 0; d < 3; d++) TRY(launch_axis_stride(ax[d], P.gm[d], GUESS_N, P.gax[d], s));
    for (int l = 0; l < P.gl; l++)
        TRY(launch_restrict<double>(P.lv[l].view64(), P.lv[l + 1].view64(), P.lv[l].b, P.lv[l + 1].b, s));
    const LevelStore& S = P.lv[P.gl];
    TRY(launch_resample(S.n, S.ax[0].c, S.ax[1].c, S.ax[2].c, S.b, G, P.gax[0], P.gax[1], P.gax[2], P.bG, 0, s));
    // faces (and a zero interior) from the fine grid's first iterate: copies at shared nodes
    const LevelStore& F = P.lv[0];
    TRY(launch_resample(F.n, F.ax[0].c, F.ax[1].c, F.ax[2].c, F.u, G, P.gax[0], P.gax[1], P.gax[2], P.fG, 0, s));
    const float* sc = guess_net_scales(h->net);
    if (lasto_nn_guess_features(G, P.bG, P.fG, P.gax[0], P.gax[1], P.gax[2], sc[0], sc[1], sc[2],
                                guess_net_features(h->net, P.gslot), s) != LASTO_OK)
        return fail(h, LASTO_ERR_CUDA, "guess features");
    return LASTO_OK;
}

// prediction -> first iterate on the fine grid (interior; faces are already set)
int enqueue_guess_out(lasto_poisson* h, ClusterPlan& P, const lasto_cluster& cl, cudaStream_t s)
{
    if (P.gl < 0) return LASTO_OK;
    const int G[3] = {GUESS_N, GUESS_N, GUESS_N};
    const float* sc = guess_net_scales(h->net);
    if (lasto_nn_guess_grid(G, guess_net_prediction(h->net, P.gslot), 16, sc[3], P.fG, P.uG, s) != LASTO_OK)
        return fail(h, LASTO_ERR_CUDA, "guess grid");
    const int gl = P.gl;
    LevelStore& S = P.lv[gl];
    const LevelStore& F = P.lv[0];
    double* tgt = gl == 0 ? P.lv[0].u : S.u;
    // coarse levels: the fine grid's faces and zero interior (copies at shared nodes)
    if (gl > 0)
        TRY(launch_resample(F.n, F.ax[0].c, F.ax[1].c, F.ax[2].c, F.u, S.n, S.ax[0].c, S.ax[1].c, S.ax[2].c, tgt, 0, s));
    TRY(launch_resample(G, P.gax[0], P.gax[1], P.gax[2], P.uG, S.n, S.ax[0].c, S.ax[1].c, S.ax[2].c, tgt, 1, s));
    for (int l = gl - 1; l >= 0; l--) {
        LevelStore& Fl = P.lv[l];
        if (l > 0)
            TRY(launch_resample(F.n, F.ax[0].c, F.ax[1].c, F.ax[2].c, F.u, Fl.n, Fl.ax[0].c, Fl.ax[1].c, Fl.ax[2].c,
                                Fl.u, 0, s));
        TRY(launch_prolong_add<double>(Fl.view64(), P.lv[l + 1].view64(), P.lv[l + 1].u, Fl.u, s));
    }
    (void)cl;
    return LASTO_OK;
}

// The mixed form with CG runs as defect correction: FP64 residual and correction
// accumulation outside, FP32 multigrid-preconditioned CG inside.
bool is_defect_correction(const lasto_poisson* h)
{
    return h->cfg.precision == LASTO_PREC_MIXED && h->cfg.cycle == LASTO_CYCLE_PCG;
}

// Measure the smoother choices of every level the cycle smooths with separate launches
// (outside any capture, once per level shape and precision; the table is kept in the handle).
int tune_plans(lasto_poisson* h, const lasto_cluster* cls, int nc, cudaStream_t s)
{
    const bool f32 = is_defect_correction(h);   // FP32 cycles run only inside defect correction
    for (int c = 0; c < nc; c++) {
        ClusterPlan& P = h->plans[c];
        int last = P.L - 2;
        if (f32) {
            const int bl = bottom_level(P);
            if (bl > 0) last = bl - 1;
        }
        bool need = false;
        for (int l = 0; l <= last; l++)
            need = need || !h->tune.count({P.lv[l].n[0], P.lv[l].n[1], P.lv[l].n[2], f32 ? 4 : 8});
        if (!need) continue;
        int st = enqueue_setup(h, P, cls[c], s);   // the level's own coefficients
        if (st) return st;
        for (int l = 0; l <= last && !st; l++)
            st = f32 ? tune_level<float>(h, P.lv[l], l == 0, s) : tune_level<double>(h, P.lv[l], l == 0, s);
        if (st) return st;
    }
    // the finest level's FP32 storage order follows its choice (fixed for every kernel of the
    // solve that touches those arrays)
    for (int c = 0; c < nc; c++) {
        ClusterPlan& P = h->plans[c];
        for (int l = 0; l < P.L; l++) P.lv[l].split32 = false;
        const int bl = bottom_level(P);
        P.lv[0].split32 = f32 && P.L >= 2 && bl != 0 && smooth_choice<float>(h, P.lv[0]).fused == 3;
    }
    return LASTO_OK;
}

// Prologue of the iteration: ||b_eff||, control block, F-cycle, starting residual.
int enqueue_start(lasto_poisson* h, ClusterPlan& P, cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s)
{
    LevelStore& F = P.lv[0];
    const LevelT<double> V = F.view64();
    const int cyc = h->cfg.cycle;
    TRY(launch_bnorm(V, F.u, F.b, P.red(FIN_BNORM), s));
    const double tol = h->cfg.rel_tol;
    const bool dc = is_defect_correction(h);
    TRY(launch_ctl_init(P.ctl, tol, (cyc == LASTO_CYCLE_PCG && !dc) ? 0.5 * tol : tol, h->cfg.max_cycles, s));
    if (cyc == LASTO_CYCLE_FV) {
        int st = enqueue_cycle<double>(h, P, 0, F.u, F.b, F.r, true, false, s);
        if (st) return st;
    }
    TRY(launch_resid_norm(V, F.u, F.b, F.r, dc ? F.b32 : nullptr, F.view32().H, P.red(FIN_START, cond, use_cond), s));
    if (cyc == LASTO_CYCLE_PCG) TRY(cudaMemsetAsync(P.p, 0, sizeof(double) * F.N(), s));
    if (dc) TRY(cudaMemsetAsync(P.e32, 0, sizeof(float) * F.N(), s));
    return LASTO_OK;
}

// One iteration (the body of the WHILE node).
int enqueue_iteration(lasto_poisson* h, ClusterPlan& P, cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s)
{
    LevelStore& F = P.lv[0];
    const LevelT<double> V = F.view64();
    if (h->cfg.cycle != LASTO_CYCLE_PCG) {
        int st = enqueue_cycle<double>(h, P, 0, F.u, F.b, F.r, false, false, s);
        if (st) return st;
        TRY(launch_resid_norm(V, F.u, F.b, F.r, nullptr, 0u, P.red(FIN_CHECK, cond, use_cond), s));
        return LASTO_OK;
    }
    TRY(cudaMemsetAsync(P.z, 0, sizeof(double) * F.N(), s));
    int st = enqueue_cycle<double>(h, P, 0, P.z, F.r, P.q, false, true, s);
    if (st) return st;
    TRY(launch_dot_rz(V, F.r, P.z, P.red(FIN_BETA), s));
    TRY(launch_update_p(V, P.ctl, P.z, P.p, s));
    TRY(launch_apply_dot(V, P.p, P.q, P.red(FIN_ALPHA), s));
    TRY(launch_update_ur(V, P.ctl, P.p, P.q, F.u, F.r, P.red(FIN_CHECK, cond, use_cond), s));
    return LASTO_OK;
}

// One FP32 CG iteration of the inner solve A e = r32 (body of the inner WHILE node).
int enqueue_inner_iteration(lasto_poisson* h, ClusterPlan& P, cudaGraphConditionalHandle cond, int use_cond,
                            cudaStream_t s)
{
    LevelStore& F = P.lv[0];
    const LevelT<float> V = F.view32();
    // the preconditioner starts from z = 0: with in-place sweeps on the finest level its first
    // red half sweep is a point update that needs no zeroed z (the faces of z were zeroed at the
    // inner solve's start, and nothing writes them); otherwise z is zeroed here
    const SmoothChoice ch0 = smooth_choice<float>(h, F);
    const int nu1_0 = h->cfg.nu_fine > 0 ? h->cfg.nu_fine : h->cfg.nu1;
    const bool point_first = P.L >= 2 && bottom_level(P) != 0 && nu1_0 >= 1 && (ch0.fused == 0 || ch0.fused == 3);
    if (!point_first) TRY(cudaMemsetAsync(F.u32, 0, sizeof(float) * F.N(), s));
    int st = enqueue_cycle<float>(h, P, 0, F.u32, F.b32, F.r32, false, true, s, point_first);
    if (st) return st;
    TRY(launch_dot32(V, F.b32, F.u32, P.red(FIN_IN_BETA), s));
    TRY(launch_update_p32(V, P.ctl, F.u32, P.p32, s));
    TRY(launch_apply_dot32(V, P.p32, P.q32, P.red(FIN_IN_ALPHA), s, P.status));
    TRY(launch_update_er32(V, P.ctl, P.p32, P.q32, P.e32, F.b32, P.red(FIN_IN_CHECK, cond, use_cond), s));
    return LASTO_OK;
}

// Start of one defect-correction step: ||r32|| and a fresh inner CG.
int enqueue_inner_start(lasto_poisson* h, ClusterPlan& P, cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s)
{
    LevelStore& F = P.lv[0];
    TRY(launch_dot32(F.view32(), F.b32, nullptr, P.red(FIN_IN_START, cond, use_cond), s));
    TRY(cudaMemsetAsync(P.p32, 0, sizeof(float) * F.N(), s));
    TRY(cudaMemsetAsync(F.u32, 0, sizeof(float) * F.N(), s));   // z, faces included
    return LASTO_OK;
}

// End of one defect-correction step: u += e in FP64, true FP64 residual (and its FP32 copy).
int enqueue_outer_finish(lasto_poisson* h, ClusterPlan& P, cudaGraphConditionalHandle cond, int use_cond,
                         cudaStream_t s)
{
    LevelStore& F = P.lv[0];
    TRY(launch_add_correction(F.N(), F.u, P.e32, F.view32().H, s));
    TRY(launch_resid_norm(F.view64(), F.u, F.b, F.r, F.b32, F.view32().H, P.red(FIN_OUTER, cond, use_cond), s));
    return LASTO_OK;
}

int enqueue_finish(lasto_poisson* h, ClusterPlan& P, const lasto_cluster& cl, double* vlm, double* potential,
                   cudaStream_t s)
{
    LevelStore& F = P.lv[0];
    const LevelT<double> V = F.view64();
    const bool dc = is_defect_correction(h);
    if (!dc) TRY(launch_resid_norm(V, F.u, F.b, nullptr, nullptr, 0u, P.red(FIN_TRUE), s));
    TRY(launch_project(cl.n, cl.x, cl.y, cl.z, F.u, cl.n_atoms, cl.pos, cl.R, h->quad, h->nq, vlm, P.status, s));
    if (potential) TRY(cudaMemcpyAsync(potential, F.u, sizeof(double) * F.N(), cudaMemcpyDeviceToDevice, s));
    k_write_stats<<<1, 1, 0, s>>>(P.ctl, P.status, P.gl >= 0 ? 1 : 0, dc ? 1 : 0, P.stats_dev);
    TRY(cudaGetLastError());
    return LASTO_OK;
}

// A conditional handle on the graph that stream s is capturing into.
int new_handle(lasto_poisson* h, cudaStream_t s, cudaGraphConditionalHandle* cond)
{
    cudaStreamCaptureStatus cstat;
    cudaGraph_t g;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cstat, nullptr, &g, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return set_cuda_error(&h->err, e, "cudaStreamGetCaptureInfo");
    e = cudaGraphConditionalHandleCreate(cond, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return set_cuda_error(&h->err, e, "cudaGraphConditionalHandleCreate");
    return LASTO_OK;
}

// A WHILE node on `cond` after everything stream s has captured so far; s continues after it.
int add_while(lasto_poisson* h, cudaStream_t s, cudaGraphConditionalHandle cond, cudaGraph_t* body)
{
    cudaStreamCaptureStatus cstat;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cstat, nullptr, &g, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return set_cuda_error(&h->err, e, "cudaStreamGetCaptureInfo");
    alignas(cudaGraphNodeParams) unsigned char cpbuf[sizeof(cudaGraphNodeParams)];
    std::memset(cpbuf, 0, sizeof(cpbuf));
    cudaGraphNodeParams* cp = reinterpret_cast<cudaGraphNodeParams*>(cpbuf);
    cp->type = cudaGraphNodeTypeConditional;
    cp->conditional.handle = cond;
    cp->conditional.type = cudaGraphCondTypeWhile;
    cp->conditional.size = 1;
    cudaGraphNode_t wnode;
    e = cudaGraphAddNode(&wnode, g, deps, nullptr, ndeps, cp);
    if (e != cudaSuccess) return set_cuda_error(&h->err, e, "cudaGraphAddNode(while)");
    *body = cp->conditional.phGraph_out[0];
    e = cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return set_cuda_error(&h->err, e, "cudaStreamUpdateCaptureDependencies");
    return LASTO_OK;
}

int count_kernels(cudaGraph_t g)
{
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    int k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        cudaGraphNodeGetType(nd, &t);
        if (t == cudaGraphNodeTypeKernel) k++;
    }
    return k;
}

// ---------------------------------------------------------------- lockstep batches (launch = 2)
// Clusters of a defect-correction batch whose hierarchies have the same shape and storage run
// their iterations in lockstep: each kernel is launched once for the whole group.
constexpr size_t LOCKSTEP_MAX = BAT_MAX;   // members per lockstep group
static_assert(sizeof(BatPack<BatLevel>) < 32000 && sizeof(BatPack<BatVec>) < 32000, "kernel parameter size");

std::vector<std::vector<int>> lockstep_groups(const lasto_poisson* h, int nc)
{
    std::vector<std::vector<int>> groups;
    if (h->cfg.launch != 2 || !is_defect_correction(h) || nc < 2) return groups;
    std::map<std::array<int, 4>, std::vector<int>> by;
    for (int c = 0; c < nc; c++) {
        const ClusterPlan& P = h->plans[c];
        if (P.L < 2 || bottom_level(P) < 1) continue;   // the group's coarsest levels run in one block
        by[{P.lv[0].n[0], P.lv[0].n[1], P.lv[0].n[2], P.lv[0].split32 ? 1 : 0}].push_back(c);
    }
    for (auto& kv : by)
        for (size_t a = 0; a < kv.second.size(); a += LOCKSTEP_MAX) {
            std::vector<int> g(kv.second.begin() + a, kv.second.begin() + std::min(kv.second.size(), a + LOCKSTEP_MAX));
            if (g.size() >= 2) groups.push_back(g);
        }
    return groups;
}

// a group's member arguments: by value for the level and vector kernels, in the handle's
// device buffer for the bottom kernel and the loop conditions
struct BatLayout {
    std::vector<BatPack<BatLevel>> lev;
    BatPack<BatVec> vec;
    size_t bot = 0, ctls = 0;
    int bl = 0;
};

BottomArgs<float> bottom_args(const lasto_poisson* h, const ClusterPlan& P, int l, bool sym)
{
    BottomArgs<float> a;
    a.nlev = P.L - l;
    for (int q = 0; q < a.nlev; q++) {
        a.lv[q] = P.lv[l + q].view32();
        a.u[q] = P.lv[l + q].u32;
        a.b[q] = P.lv[l + q].b32;
    }
    a.eig = P.eig;
    a.nu1 = h->cfg.nu_coarse;
    a.nu2 = h->cfg.nu_coarse;
    a.sym = sym ? 1 : 0;
    return a;
}

// Fill the groups' argument arrays and copy them to the device (outside any capture).
int upload_bat_args(lasto_poisson* h, const std::vector<std::vector<int>>& groups, std::vector<BatLayout>& lay)
{
    std::vector<char> blob;
    auto put = [&](const void* src, size_t bytes) {
        const size_t off = (blob.size() + 255) & ~size_t(255);
        blob.resize(off + bytes);
        std::memcpy(blob.data() + off, src, bytes);
        return off;
    };
    lay.assign(groups.size(), BatLayout());
    for (size_t gi = 0; gi < groups.size(); gi++) {
        const std::vector<int>& g = groups[gi];
        const int nm = (int)g.size();
        BatLayout& L = lay[gi];
        if (nm > BAT_MAX) return fail(h, LASTO_ERR_INVALID_ARG, "lockstep group too large");
        L.bl = bottom_level(h->plans[g[0]]);
        L.lev.assign(L.bl, BatPack<BatLevel>());
        std::memset(L.lev.data(), 0, sizeof(BatPack<BatLevel>) * L.lev.size());
        for (int l = 0; l < L.bl; l++) {
            for (int q = 0; q < nm; q++) {
                const ClusterPlan& P = h->plans[g[q]];
                BatLevel& v = L.lev[l].m[q];
                v.V = P.lv[l].view32();
                v.VC = P.lv[l + 1].view32();
                v.u = P.lv[l].u32;
                v.b = P.lv[l].b32;
                v.uc = P.lv[l + 1].u32;
                v.bc = P.lv[l + 1].b32;
                v.ctl = P.ctl;
            }
        }
        std::memset(&L.vec, 0, sizeof(L.vec));
        std::vector<BatBottom> bb(nm);
        std::vector<Ctl*> cc(nm);
        for (int q = 0; q < nm; q++) {
            const ClusterPlan& P = h->plans[g[q]];
            const LevelStore& F = P.lv[0];
            bb[q].a = bottom_args(h, P, L.bl, true);
            bb[q].ctl = P.ctl;
            BatVec& a = L.vec.m[q];
            a.V32 = F.view32();
            a.V64 = F.view64();
            a.u32 = F.u32;
            a.b32 = F.b32;
            a.e32 = P.e32;
            a.p32 = P.p32;
            a.q32 = P.q32;
            a.u = F.u;
            a.b = F.b;
            a.r = F.r;
            a.part = P.part;
            a.counter = reinterpret_cast<unsigned int*>(P.status + 1);
            a.ctl = P.ctl;
            a.status = P.status;
            cc[q] = P.ctl;
        }
        L.bot = put(bb.data(), sizeof(BatBottom) * nm);
        L.ctls = put(cc.data(), sizeof(Ctl*) * nm);
    }
    if (blob.empty()) return LASTO_OK;
    if (blob.size() > h->bat_bytes) {
        if (h->bat_args) cudaFree(h->bat_args);
        h->bat_args = nullptr;
        h->bat_bytes = 0;
        TRY(cudaMalloc(&h->bat_args, blob.size()));
        h->bat_bytes = blob.size();
    }
    TRY(cudaMemcpy(h->bat_args, blob.data(), blob.size(), cudaMemcpyHostToDevice));
    return LASTO_OK;
}

// One FP32 V-cycle of every member of a group (the preconditioner of the inner CG: symmetric
// smoothing order), levels 0 .. bl-1 launched, the rest in one block per member.
int enqueue_cycle_bat(lasto_poisson* h, const std::vector<int>& g, const BatLayout& L, cudaStream_t s)
{
    const ClusterPlan& P = h->plans[g[0]];
    const int nm = (int)g.size();
    auto lev = [&](int l) -> const BatPack<BatLevel>& { return L.lev[l]; };
    auto nu_of = [&](int l, int v) { return (l == 0 && h->cfg.nu_fine > 0) ? h->cfg.nu_fine : v; };
    auto nt_of = [&](int l) {
        const SmoothChoice ch = smooth_choice<float>(h, P.lv[l]);
        return ((ch.fused == 0 || ch.fused == 3) && ch.nt >= 32) ? ch.nt : 256;
    };
    for (int l = 0; l < L.bl; l++) {
        const LevelT<float> V = P.lv[l].view32(), VC = P.lv[l + 1].view32();
        const int nu1 = nu_of(l, h->cfg.nu1), nt = nt_of(l);
        for (int it = 0; it < nu1; it++) {
            TRY(launch_rbgs_bat(V, lev(l), nm, 0, nt, s));
            TRY(launch_rbgs_bat(V, lev(l), nm, 1, nt, s));
        }
        // after nu1 >= 1 sweeps that end on the black half sweep the black residuals are zero
        TRY(launch_resid_restrict_bat(V, VC, lev(l), nm, nu1 > 0, s));
    }
    TRY(launch_bottom_bat(bottom_args(h, P, L.bl, true), reinterpret_cast<const BatBottom*>(h->bat_args + L.bot), nm,
                          s));
    for (int l = L.bl - 1; l >= 0; l--) {
        const LevelT<float> V = P.lv[l].view32(), VC = P.lv[l + 1].view32();
        const int nu2 = nu_of(l, h->cfg.nu2), nt = nt_of(l);
        TRY(launch_prolong_add_bat(V, VC, lev(l), nm, s));
        for (int it = 0; it < nu2; it++) {
            TRY(launch_rbgs_bat(V, lev(l), nm, 1, nt, s));
            TRY(launch_rbgs_bat(V, lev(l), nm, 0, nt, s));
        }
    }
    return LASTO_OK;
}

// The defect-correction loops of one group, captured on stream gs: the outer WHILE over the
// members' FP64 corrections around the inner WHILE of their FP32 CG iterations.
int capture_group_loops(lasto_poisson* h, const std::vector<int>& g, const BatLayout& L, cudaStream_t gs)
{
    const ClusterPlan& P = h->plans[g[0]];
    const int nm = (int)g.size();
    const LevelStore& F = P.lv[0];
    const LevelT<float> V32 = F.view32();
    const BatPack<BatVec>& vec = L.vec;
    Ctl* const* ctls = reinterpret_cast<Ctl* const*>(h->bat_args + L.ctls);
    cudaGraphConditionalHandle cout_;
    int st = new_handle(h, gs, &cout_);
    if (st) return st;
    TRY(launch_any_bat(ctls, nm, BAT_OUTER, cout_, gs));
    cudaGraph_t body;
    if ((st = add_while(h, gs, cout_, &body))) return st;
    cudaError_t e = cudaStreamBeginCaptureToGraph(h->cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return set_cuda_error(&h->err, e, "cudaStreamBeginCaptureToGraph");
    h->outer_bodies.push_back(body);
    auto outer = [&]() -> int {
        TRY(launch_dot32_bat(V32, vec, nm, 0, FIN_IN_START, BAT_OUTER, h->cs2));
        TRY(launch_zero_bat(vec, nm, F.N(), 1, BAT_OUTER, h->cs2));
        cudaGraphConditionalHandle cin;
        int r = new_handle(h, h->cs2, &cin);
        if (r) return r;
        TRY(launch_any_bat(ctls, nm, BAT_INNER, cin, h->cs2));
        cudaGraph_t ibody;
        if ((r = add_while(h, h->cs2, cin, &ibody))) return r;
        h->bodies.push_back(ibody);
        cudaError_t e2 = cudaStreamBeginCaptureToGraph(h->cs3, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e2 != cudaSuccess) return set_cuda_error(&h->err, e2, "cudaStreamBeginCaptureToGraph(inner)");
        auto inner = [&]() -> int {
            TRY(launch_zero_bat(vec, nm, F.N(), 0, BAT_INNER, h->cs3));
            int q = enqueue_cycle_bat(h, g, L, h->cs3);
            if (q) return q;
            TRY(launch_dot32_bat(V32, vec, nm, 1, FIN_IN_BETA, BAT_INNER, h->cs3));
            TRY(launch_update_p32_bat(V32, vec, nm, h->cs3));
            TRY(launch_apply_dot32_bat(V32, vec, nm, h->cs3));
            TRY(launch_update_er32_bat(V32, vec, nm, h->cs3));
            TRY(launch_any_bat(ctls, nm, BAT_INNER, cin, h->cs3));
            return LASTO_OK;
        };
        r = inner();
        cudaGraph_t iout = nullptr;
        e2 = cudaStreamEndCapture(h->cs3, &iout);
        if (r) return r;
        if (e2 != cudaSuccess) return set_cuda_error(&h->err, e2, "cudaStreamEndCapture(inner)");
        TRY(launch_outer_bat(F.view64(), vec, nm, V32.H, h->cs2));
        TRY(launch_any_bat(ctls, nm, BAT_OUTER, cout_, h->cs2));
        return LASTO_OK;
    };
    st = outer();
    cudaGraph_t bout = nullptr;
    e = cudaStreamEndCapture(h->cs2, &bout);
    if (st) return st;
    if (e != cudaSuccess) return set_cuda_error(&h->err, e, "cudaStreamEndCapture(body)");
    return LASTO_OK;
}

int capture_solve(lasto_poisson* h, const lasto_cluster* cls, int nc, double* v_lm, double* potential,
                  const double* guess)
{
    cudaStream_t s = h->cs;
    h->bodies.clear();
    h->outer_bodies.clear();
    const std::vector<std::vector<int>> groups = lockstep_groups(h, nc);
    std::vector<BatLayout> lay;
    if (int r = upload_bat_args(h, groups, lay)) return r;
    std::vector<int> group_of(nc, -1);
    for (size_t gi = 0; gi < groups.size(); gi++)
        for (int c : groups[gi]) group_of[c] = (int)gi;
    std::vector<size_t> atom_offs(nc, 0), grid_offs(nc, 0);
    for (int c = 1; c < nc; c++) {
        atom_offs[c] = atom_offs[c - 1] + cls[c - 1].n_atoms;
        grid_offs[c] = grid_offs[c - 1] + (size_t)cls[c - 1].n[0] * cls[c - 1].n[1] * cls[c - 1].n[2];
    }
    TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int st = LASTO_OK;
    size_t atom_off = 0, grid_off = 0;
    // every cluster is an independent branch of the graph: small clusters' latency-bound
    // kernels run side by side instead of one after another.  With the learned guess the
    // branches join once, after every right-hand side, for one batched network pass.
    const int nguess = plan_guesses(h, cls, nc, guess);
    if (cudaEventRecord(h->ev_origin, s) != cudaSuccess) st = LASTO_ERR_CUDA;
    for (int c = 0; c < nc && st == LASTO_OK; c++) {
        ClusterPlan& P = h->plans[c];
        cudaStream_t bsc = h->bs[c];
        cudaError_t e = cudaStreamWaitEvent(bsc, h->ev_origin, 0);
        if (e != cudaSuccess) { st = set_cuda_error(&h->err, e, "cudaStreamWaitEvent(origin)"); break; }
        if ((st = enqueue_prologue(h, P, cls[c], guess ? guess + grid_off : nullptr, bsc, c))) break;
        grid_off += (size_t)cls[c].n[0] * cls[c].n[1] * cls[c].n[2];
        if (nguess > 0) {
            if ((st = enqueue_guess_in(h, P, cls[c], bsc))) break;
            e = cudaEventRecord(h->eg[c], bsc);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->eg[c], 0);
            if (e != cudaSuccess) { st = set_cuda_error(&h->err, e, "guess join"); break; }
        }
    }
    if (st == LASTO_OK && nguess > 0) {
        st = guess_net_forward(h->net, nguess, s);
        if (st) fail(h, st, "guess network forward");
        else if (cudaEventRecord(h->ev_net, s) != cudaSuccess) st = fail(h, LASTO_ERR_CUDA, "guess fork");
    }
    grid_off = 0;
    for (int c = 0; c < nc && st == LASTO_OK; c++) {
        ClusterPlan& P = h->plans[c];
        const lasto_cluster& cl = cls[c];
        cudaStream_t bsc = h->bs[c];
        cudaError_t e;
        if (nguess > 0) {
            e = cudaStreamWaitEvent(bsc, h->ev_net, 0);
            if (e != cudaSuccess) { st = set_cuda_error(&h->err, e, "guess fork"); break; }
            if ((st = enqueue_guess_out(h, P, cl, bsc))) break;
        }
        if (group_of[c] >= 0) {
            // a lockstep member: its loops run with its group's (below)
            if ((st = enqueue_start(h, P, 0, 0, bsc))) break;
            e = cudaEventRecord(h->es[c], bsc);
            if (e != cudaSuccess) { st = set_cuda_error(&h->err, e, "lockstep start"); break; }
            atom_off += cl.n_atoms;
            grid_off += (size_t)cl.n[0] * cl.n[1] * cl.n[2];
            continue;
        }
        // conditional WHILE node(s) for the iteration
        cudaGraphConditionalHandle cond;
        if ((st = new_handle(h, bsc, &cond))) break;
        if ((st = enqueue_start(h, P, cond, 1, bsc))) break;
        cudaGraph_t body;
        if ((st = add_while(h, bsc, cond, &body))) break;
        e = cudaStreamBeginCaptureToGraph(h->cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { st = set_cuda_error(&h->err, e, "cudaStreamBeginCaptureToGraph"); break; }
        if (is_defect_correction(h)) {
            // outer body: inner start, inner WHILE (FP32 CG), FP64 correction + residual
            h->outer_bodies.push_back(body);
            cudaGraphConditionalHandle cin;
            cudaGraph_t ibody;
            st = new_handle(h, h->cs2, &cin);
            if (!st) st = enqueue_inner_start(h, P, cin, 1, h->cs2);
            if (!st) st = add_while(h, h->cs2, cin, &ibody);
            if (!st) {
                h->bodies.push_back(ibody);
                e = cudaStreamBeginCaptureToGraph(h->cs3, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) st = set_cuda_error(&h->err, e, "cudaStreamBeginCaptureToGraph(inner)");
                else {
                    st = enqueue_inner_iteration(h, P, cin, 1, h->cs3);
                    cudaGraph_t iout = nullptr;
                    e = cudaStreamEndCapture(h->cs3, &iout);
                    if (!st && e != cudaSuccess) st = set_cuda_error(&h->err, e, "cudaStreamEndCapture(inner)");
                }
            }
            if (!st) st = enqueue_outer_finish(h, P, cond, 1, h->cs2);
        } else {
            h->bodies.push_back(body);
            st = enqueue_iteration(h, P, cond, 1, h->cs2);
        }
        cudaGraph_t bout = nullptr;
        e = cudaStreamEndCapture(h->cs2, &bout);
        if (st) break;
        if (e != cudaSuccess) { st = set_cuda_error(&h->err, e, "cudaStreamEndCapture(body)"); break; }
        if ((st = enqueue_finish(h, P, cl, v_lm + NLM * atom_off, potential ? potential + grid_off : nullptr, bsc)))
            break;
        e = cudaEventRecord(h->ed[c], bsc);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ed[c], 0);
        if (e != cudaSuccess) { st = set_cuda_error(&h->err, e, "join"); break; }
        atom_off += cl.n_atoms;
        grid_off += (size_t)cl.n[0] * cl.n[1] * cl.n[2];
    }
    for (size_t gi = 0; gi < groups.size() && st == LASTO_OK; gi++) {
        const std::vector<int>& grp = groups[gi];
        cudaStream_t gs = h->bs[grp[0]];
        cudaError_t e = cudaSuccess;
        for (int c : grp)
            if (e == cudaSuccess && c != grp[0]) e = cudaStreamWaitEvent(gs, h->es[c], 0);
        if (e != cudaSuccess) { st = set_cuda_error(&h->err, e, "lockstep join"); break; }
        if ((st = capture_group_loops(h, grp, lay[gi], gs))) break;
        if ((e = cudaEventRecord(h->eb[grp[0]], gs)) != cudaSuccess) { st = set_cuda_error(&h->err, e, "lockstep fork"); break; }
        for (int c : grp) {
            cudaStream_t bsc = h->bs[c];
            if (c != grp[0] && (e = cudaStreamWaitEvent(bsc, h->eb[grp[0]], 0)) != cudaSuccess) {
                st = set_cuda_error(&h->err, e, "lockstep fork");
                break;
            }
            if ((st = enqueue_finish(h, h->plans[c], cls[c], v_lm + NLM * atom_offs[c],
                                     potential ? potential + grid_offs[c] : nullptr, bsc)))
                break;
            e = cudaEventRecord(h->ed[c], bsc);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ed[c], 0);
            if (e != cudaSuccess) { st = set_cuda_error(&h->err, e, "join"); break; }
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return set_cuda_error(&h->err, e, "cudaStreamEndCapture");
    {
        // kernel nodes of the top-level graph and of the WHILE bodies
        h->kernels_fixed = count_kernels(g);
        int it = 0, ou = 0;
        for (cudaGraph_t bg : h->bodies) it += count_kernels(bg);
        for (cudaGraph_t bg : h->outer_bodies) ou += count_kernels(bg);
        h->kernels_iter = h->bodies.empty() ? 0 : it / (int)h->bodies.size();
        h->kernels_outer = h->outer_bodies.empty() ? 0 : ou / (int)h->outer_bodies.size();
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return set_cuda_error(&h->err, e, "cudaGraphInstantiate");
    }
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->graph = g;
    h->exec = ex;
    return LASTO_OK;
}

// One solve's stats, from the pinned staging buffer to the caller's array.  Each call carries
// its own destination, so solves enqueued back to back on one handle (before the first has
// finished) each fill their own array; the staging buffer is reused in stream order.
struct StatsCopy {
    lasto_stats* dst;
    const lasto_stats* src;
    int count;
};

void CUDART_CB copy_stats_out(void* arg)
{
    StatsCopy* c = static_cast<StatsCopy*>(arg);
    std::memcpy(c->dst, c->src, sizeof(lasto_stats) * c->count);
    delete c;
}

}  // namespace

static int copy_stats(lasto_poisson* h, int nc, lasto_stats* stats, cudaStream_t s)
{
    cudaError_t e;
    if (stats) {
        for (int c = 0; c < nc; c++) {
            e = cudaMemcpyAsync(h->stats_pinned + c, h->plans[c].stats_dev, sizeof(lasto_stats),
                                cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return set_cuda_error(&h->err, e, "stats copy");
        }
        StatsCopy* c = new StatsCopy{stats, h->stats_pinned, nc};
        e = cudaLaunchHostFunc(s, copy_stats_out, c);
        if (e != cudaSuccess) {
            delete c;
            return set_cuda_error(&h->err, e, "cudaLaunchHostFunc");
        }
    }
    return LASTO_OK;
}

// The same kernels as the captured graph, launched directly; the iteration loop runs
// on the host and reads the device control block once per iteration.
static int direct_solve(lasto_poisson* h, const lasto_cluster* cls, const lasto_raw_cluster* raws, int nc,
                        double* v_lm, double* potential, const double* guess, cudaStream_t s)
{
    h->plans.assign(nc, ClusterPlan());
    h->key.clear();
    Carver cv{h->pool, h->pool_bytes};
    for (int c = 0; c < nc; c++) {
        if (!carve_cluster(cv, cls[c].n, cls[c].n_atoms, h->plans[c]))
            return fail(h, LASTO_ERR_NO_MEMORY, "workspace too small for this batch");
        h->plans[c].raw = raws ? raws + c : nullptr;
    }
    {
        NvtxRange r("lasto: smoother tuning");
        if (int st = tune_plans(h, cls, nc, s)) return st;
    }
    size_t atom_off = 0, grid_off = 0;
    const int nguess = plan_guesses(h, cls, nc, guess);
    for (int c = 0; c < nc; c++) {
        NvtxRange r("lasto: deposit, multipoles, faces");
        int st;
        if ((st = enqueue_prologue(h, h->plans[c], cls[c], guess ? guess + grid_off : nullptr, s, 0))) return st;
        if ((st = enqueue_guess_in(h, h->plans[c], cls[c], s))) return st;
        grid_off += (size_t)cls[c].n[0] * cls[c].n[1] * cls[c].n[2];
    }
    if (nguess > 0) {
        NvtxRange r("lasto: learned guess");
        const int st = guess_net_forward(h->net, nguess, s);
        if (st) return fail(h, st, "guess network forward");
    }
    grid_off = 0;
    for (int c = 0; c < nc; c++) {
        NvtxRange r("lasto: iteration");
        ClusterPlan& P = h->plans[c];
        const lasto_cluster& cl = cls[c];
        int st;
        if ((st = enqueue_guess_out(h, P, cl, s))) return st;
        if ((st = enqueue_start(h, P, 0, 0, s))) return st;
        int done = 0;
        TRY(cudaMemcpyAsync(&done, &P.ctl->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        TRY(cudaStreamSynchronize(s));
        if (is_defect_correction(h)) {
            for (int outer = 0; outer < h->cfg.max_cycles && !done; outer++) {
                if ((st = enqueue_inner_start(h, P, 0, 0, s))) return st;
                int go = 0;
                TRY(cudaMemcpyAsync(&go, &P.ctl->go_in, sizeof(int), cudaMemcpyDeviceToHost, s));
                TRY(cudaStreamSynchronize(s));
                while (go) {
                    if ((st = enqueue_inner_iteration(h, P, 0, 0, s))) return st;
                    TRY(cudaMemcpyAsync(&go, &P.ctl->go_in, sizeof(int), cudaMemcpyDeviceToHost, s));
                    TRY(cudaStreamSynchronize(s));
                }
                if ((st = enqueue_outer_finish(h, P, 0, 0, s))) return st;
                TRY(cudaMemcpyAsync(&done, &P.ctl->done, sizeof(int), cudaMemcpyDeviceToHost, s));
                TRY(cudaStreamSynchronize(s));
            }
        } else {
            for (int it = 0; it < h->cfg.max_cycles && !done; it++) {
                if ((st = enqueue_iteration(h, P, 0, 0, s))) return st;
                TRY(cudaMemcpyAsync(&done, &P.ctl->done, sizeof(int), cudaMemcpyDeviceToHost, s));
                TRY(cudaStreamSynchronize(s));
            }
        }
        NvtxRange rf("lasto: projection");
        if ((st = enqueue_finish(h, P, cl, v_lm + NLM * atom_off, potential ? potential + grid_off : nullptr, s)))
            return st;
        atom_off += cl.n_atoms;
        grid_off += (size_t)cl.n[0] * cl.n[1] * cl.n[2];
    }
    return LASTO_OK;
}

// ================================================================ ABI
extern "C" {

void lasto_config_default(lasto_config* c)
{
    if (!c) return;
    c->n_max = 129;
    c->max_atoms = 561;
    c->max_batch = 1;
    c->precision = LASTO_PREC_FP64;
    c->cycle = LASTO_CYCLE_PCG;
    c->nu1 = 4;
    c->nu2 = 4;
    c->max_cycles = 50;
    c->rel_tol = 1e-10;
    c->n_theta = 16;
    c->n_phi = 32;
    c->launch = 0;
    c->boundary = LASTO_BC_MULTIPOLE;
    c->nu_coarse = 4;
    c->nu_fine = 0;
}

int lasto_poisson_create(const lasto_config* cfg, lasto_poisson** out)
{
    if (!out) return LASTO_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg) return LASTO_ERR_INVALID_ARG;
    const int nm[3] = {cfg->n_max, cfg->n_max, cfg->n_max};
    if (!valid_n(nm) || cfg->max_atoms < 1 || cfg->max_batch < 1 || cfg->nu1 < 0 || cfg->nu2 < 0 ||
        cfg->nu1 + cfg->nu2 < 1 || cfg->max_cycles < 1 || cfg->max_cycles >= CTL_HIST || !(cfg->rel_tol > 0.0) ||
        cfg->n_theta < 1 || cfg->n_theta > 32 || cfg->n_phi < 1 || cfg->n_phi > 64 ||
        (cfg->precision != LASTO_PREC_FP64 && cfg->precision != LASTO_PREC_MIXED) ||
        (cfg->cycle != LASTO_CYCLE_V && cfg->cycle != LASTO_CYCLE_FV && cfg->cycle != LASTO_CYCLE_PCG) ||
        (cfg->launch < 0 || cfg->launch > 2) || cfg->nu_coarse < 0 || cfg->nu_coarse > 64 || cfg->nu_fine < 0 || cfg->nu_fine > 64 ||
        (cfg->boundary != LASTO_BC_MULTIPOLE && cfg->boundary != LASTO_BC_ZERO && cfg->boundary != LASTO_BC_EXACT))
        return LASTO_ERR_INVALID_ARG;
    lasto_poisson* h = new (std::nothrow) lasto_poisson();
    if (!h) return LASTO_ERR_NO_MEMORY;
    h->cfg = *cfg;
    cudaGetDevice(&h->device);
    init_device_constants();
    const size_t per = cluster_bytes(nm, cfg->max_atoms);
    h->pool_bytes = per * (size_t)cfg->max_batch;
    cudaError_t e = cudaMalloc(&h->pool, h->pool_bytes);
    if (e != cudaSuccess) {
        delete h;
        return e == cudaErrorMemoryAllocation ? LASTO_ERR_NO_MEMORY : LASTO_ERR_CUDA;
    }
    h->nq = cfg->n_theta * cfg->n_phi;
    std::vector<double> tab((size_t)h->nq * 28);
    host_quadrature(cfg->n_theta, cfg->n_phi, tab.data());
    e = cudaMalloc(&h->quad, sizeof(double) * tab.size());
    if (e == cudaSuccess) e = cudaMemcpy(h->quad, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cs2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cs3, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_origin, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_net, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_launch, cudaEventDisableTiming);
    h->bs.assign(cfg->max_batch, nullptr);
    h->ss.assign(cfg->max_batch, nullptr);
    h->ef.assign(cfg->max_batch, nullptr);
    h->ej.assign(cfg->max_batch, nullptr);
    h->ed.assign(cfg->max_batch, nullptr);
    h->eg.assign(cfg->max_batch, nullptr);
    h->es.assign(cfg->max_batch, nullptr);
    h->eb.assign(cfg->max_batch, nullptr);
    for (int c = 0; c < cfg->max_batch && e == cudaSuccess; c++) {
        e = cudaStreamCreateWithFlags(&h->bs[c], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->ss[c], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ef[c], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ej[c], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ed[c], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->eg[c], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->es[c], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->eb[c], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMallocHost(&h->stats_pinned, sizeof(lasto_stats) * cfg->max_batch);
    if (e != cudaSuccess) {
        lasto_poisson_destroy(h);
        return LASTO_ERR_CUDA;
    }
    *out = h;
    return LASTO_OK;
}

void lasto_poisson_destroy(lasto_poisson* h)
{
    if (!h) return;
    if (h->ev_launch) cudaEventSynchronize(h->ev_launch);   // the last solve and its stats copy
    if (h->cs) cudaStreamSynchronize(h->cs);
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->pool) cudaFree(h->pool);
    if (h->quad) cudaFree(h->quad);
    if (h->stats_pinned) cudaFreeHost(h->stats_pinned);
    if (h->cs) cudaStreamDestroy(h->cs);
    if (h->cs2) cudaStreamDestroy(h->cs2);
    if (h->cs3) cudaStreamDestroy(h->cs3);
    if (h->ev_origin) cudaEventDestroy(h->ev_origin);
    for (auto x : h->bs) if (x) cudaStreamDestroy(x);
    for (auto x : h->ss) if (x) cudaStreamDestroy(x);
    for (auto x : h->ef) if (x) cudaEventDestroy(x);
    for (auto x : h->ej) if (x) cudaEventDestroy(x);
    for (auto x : h->ed) if (x) cudaEventDestroy(x);
    for (auto x : h->eg) if (x) cudaEventDestroy(x);
    for (auto x : h->es) if (x) cudaEventDestroy(x);
    for (auto x : h->eb) if (x) cudaEventDestroy(x);
    if (h->bat_args) cudaFree(h->bat_args);
    if (h->ev_net) cudaEventDestroy(h->ev_net);
    if (h->ev_launch) cudaEventDestroy(h->ev_launch);
    guess_net_free(h->net);
    delete h;
}

int lasto_poisson_kernel_counts(const lasto_poisson* h, int* fixed, int* per_iteration, int* per_outer)
{
    if (!h || !fixed || !per_iteration || !per_outer || h->kernels_fixed < 0) return LASTO_ERR_INVALID_ARG;
    *fixed = h->kernels_fixed;
    *per_iteration = h->kernels_iter;
    *per_outer = h->kernels_outer;
    return LASTO_OK;
}

int lasto_poisson_tune_table(const lasto_poisson* h, char* buf, size_t cap)
{
    if (!h) return -1;
    std::string out;
    char line[160];
    for (const auto& kv : h->tune) {
        const SmoothChoice& c = kv.second;
        std::snprintf(line, sizeof(line), "%d %d %d %d %d %d %d %d %d %d %.3f\n", kv.first[0], kv.first[1], kv.first[2],
                      kv.first[3], c.fused, c.nt, c.sh.tx, c.sh.ty, c.sh.kz, c.sh.ns, (double)c.us);
        out += line;
    }
    if (buf && cap > 0) {
        const size_t n = std::min(cap - 1, out.size());
        std::memcpy(buf, out.data(), n);
        buf[n] = '\0';
    }
    return (int)out.size();
}

int lasto_poisson_set_tune_table(lasto_poisson* h, const char* text)
{
    if (!h || !text) return LASTO_ERR_INVALID_ARG;
    std::map<std::array<int, 4>, SmoothChoice> add;
    const char* p = text;
    for (;;) {
        while (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t') p++;
        if (!*p) break;
        std::array<int, 4> k{};
        SmoothChoice c;
        double us = 0.0;
        int used = 0;
        const int got = std::sscanf(p, "%d %d %d %d %d %d %d %d %d %d %lf%n", &k[0], &k[1], &k[2], &k[3], &c.fused,
                                    &c.nt, &c.sh.tx, &c.sh.ty, &c.sh.kz, &c.sh.ns, &us, &used);
        if (got < 11 || used <= 0) return fail(h, LASTO_ERR_INVALID_ARG, "tune table line");
        c.us = (float)us;
        if ((k[3] != 4 && k[3] != 8) || !choice_usable(h, c, (size_t)k[3]))
            return fail(h, LASTO_ERR_INVALID_ARG, "tune table entry");
        add[k] = c;
        p += used;
    }
    for (const auto& kv : add) h->tune[kv.first] = kv.second;
    h->key.clear();   // recapture with the new choices
    return LASTO_OK;
}

size_t lasto_guess_param_count(void) { return guess_param_count(); }

int lasto_poisson_set_guess(lasto_poisson* h, const float* params, size_t n_params, const double scales[4])
{
    if (!h) return LASTO_ERR_INVALID_ARG;
    if (h->cs) cudaStreamSynchronize(h->cs);
    GuessNet* g = nullptr;
    if (params) {
        const int st = guess_net_create(params, n_params, scales, h->cfg.max_batch, &g, h->cs);
        if (st) return fail(h, st, "guess network");
    }
    guess_net_free(h->net);
    h->net = g;
    h->key.clear();   // the cached graph was captured without (or with another) network
    return LASTO_OK;
}

const char* lasto_poisson_last_error(const lasto_poisson* h)
{
    return h ? h->err.msg.c_str() : "null handle";
}

static int solve_impl(lasto_poisson* h, const lasto_cluster* cls, const lasto_raw_cluster* raws, int nc,
                      double* v_lm, double* potential, const double* guess, lasto_stats* stats, void* stream)
{
    if (!h) return LASTO_ERR_INVALID_ARG;
    NvtxRange range("lasto_poisson_solve");
    h->err = Err();
    if (!cls || nc < 1 || nc > h->cfg.max_batch || !v_lm) return fail(h, LASTO_ERR_INVALID_ARG, "bad clusters/outputs");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // key of the captured graph: every pointer and size the graph bakes in
    std::vector<char> key;
    auto put = [&](const void* p, size_t n) {
        const char* c = static_cast<const char*>(p);
        key.insert(key.end(), c, c + n);
    };
    for (int c = 0; c < nc; c++) {
        const lasto_cluster& cl = cls[c];
        if (!valid_n(cl.n) || cl.n[0] > h->cfg.n_max || cl.n[1] > h->cfg.n_max || cl.n[2] > h->cfg.n_max)
            return fail(h, LASTO_ERR_INVALID_ARG, "grid size: odd, >= 3, coarsening to <= 9 nodes, <= n_max");
        if (cl.n_atoms < 1 || cl.n_atoms > h->cfg.max_atoms || !cl.pos || !cl.Z || !cl.R || !cl.x || !cl.y || !cl.z)
            return fail(h, LASTO_ERR_INVALID_ARG, "cluster arrays");
        if (raws) {
            const lasto_raw_cluster& r = raws[c];
            if (!r.density || !r.rho00 || r.n_rad < 5 || !(r.r_min > 0.0))
                return fail(h, LASTO_ERR_INVALID_ARG, "raw density arrays");
            if (h->cfg.boundary == LASTO_BC_EXACT)
                return fail(h, LASTO_ERR_INVALID_ARG, "exact faces need the model density");
            put(&r, sizeof(r));
        } else if (!cl.slater_w || !cl.slater_zeta || !cl.c_lm) {
            return fail(h, LASTO_ERR_INVALID_ARG, "cluster arrays");
        }
        put(&cl, sizeof(cl));
    }
    put(&v_lm, sizeof(v_lm));
    put(&potential, sizeof(potential));
    put(&guess, sizeof(guess));
    put(&nc, sizeof(nc));
    if (h->cfg.launch == 1) {
        TRY(cudaEventSynchronize(h->ev_launch));
        int st = direct_solve(h, cls, raws, nc, v_lm, potential, guess, s);
        if (!st) st = copy_stats(h, nc, stats, s);
        if (!st) TRY(cudaEventRecord(h->ev_launch, s));
        return st;
    }
    if (key != h->key || !h->exec) {
        // a solve launched earlier (possibly still running) uses the workspace and the graph
        TRY(cudaEventSynchronize(h->ev_launch));
        // carve the workspace for these clusters
        h->plans.assign(nc, ClusterPlan());
        Carver cv{h->pool, h->pool_bytes};
        for (int c = 0; c < nc; c++) {
            if (!carve_cluster(cv, cls[c].n, cls[c].n_atoms, h->plans[c]))
                return fail(h, LASTO_ERR_NO_MEMORY, "workspace too small for this batch");
            h->plans[c].raw = raws ? raws + c : nullptr;
        }
        h->key.clear();
        int st;
        {
            NvtxRange r("lasto: smoother tuning");
            st = tune_plans(h, cls, nc, s);
        }
        if (st) return st;
        {
            NvtxRange r("lasto: graph capture");
            st = capture_solve(h, cls, nc, v_lm, potential, guess);
        }
        if (st) return st;
        h->key = key;
        h->n_clusters = nc;
    }
    NvtxRange rl("lasto: graph launch");
    cudaError_t e = cudaGraphLaunch(h->exec, s);
    if (e != cudaSuccess) return set_cuda_error(&h->err, e, "cudaGraphLaunch");
    const int st = copy_stats(h, nc, stats, s);
    if (st) return st;
    TRY(cudaEventRecord(h->ev_launch, s));
    return LASTO_OK;
}

extern "C" int lasto_poisson_solve(lasto_poisson* h, const lasto_cluster* cls, int nc, double* v_lm, double* potential,
                                   const double* guess, lasto_stats* stats, void* stream)
{
    return solve_impl(h, cls, nullptr, nc, v_lm, potential, guess, stats, stream);
}

extern "C" int lasto_poisson_solve_raw(lasto_poisson* h, const lasto_raw_cluster* raws, int nc, double* v_lm,
                                       double* potential, const double* guess, lasto_stats* stats, void* stream)
{
    if (!h) return LASTO_ERR_INVALID_ARG;
    if (!raws || nc < 1 || nc > h->cfg.max_batch) return fail(h, LASTO_ERR_INVALID_ARG, "bad clusters");
    std::vector<lasto_cluster> cls(nc);
    for (int c = 0; c < nc; c++) cls[c] = cluster_of(raws[c]);
    // the raw structs must outlive the capture only: the graph keeps copies of their values
    h->raw_copy.assign(raws, raws + nc);
    return solve_impl(h, cls.data(), h->raw_copy.data(), nc, v_lm, potential, guess, stats, stream);
}

// ---------------------------------------------------------------- mesh
int lasto_mesh_axis(int n, double centre, double half_width, double h_min, double h_max, double p_max, double* x,
                    double* info, void* stream)
{
    if (n < 3 || n % 2 == 0 || !x || !(half_width > 0.0) || !(h_min > 0.0) || !(h_max > 0.0)) return LASTO_ERR_INVALID_ARG;
    const double m = 0.5 * (n - 1);
    const double A = h_min * m, B = half_width - A;
    if (B < -1e-12 * half_width) return LASTO_ERR_INVALID_ARG;
    if (B > 1e-12 * half_width) {
        double p = (h_max * m - A) / B;
        double AA = A;
        if (p > p_max) {
            if (!(p_max > 1.0)) return LASTO_ERR_INVALID_ARG;
            const double BB = (h_max * m - half_width) / (p_max - 1.0);
            AA = half_width - BB;
            p = p_max;
        }
        if (!(p >= 1.0) || !(AA > 0.0)) return LASTO_ERR_INVALID_ARG;
    }
    cudaError_t e = launch_mesh_axis(n, centre, half_width, h_min, h_max, p_max, x, info, (cudaStream_t)stream);
    return e == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA;
}

}  // extern "C"

// ================================================================ single operations
namespace {

// Level tables (and optional inverse diagonal) for one grid in scratch memory.
struct OpLevel {
    Scratch mem;
    LevelStore S;
    OpLevel(const int n[3], const double* x, const double* y, const double* z, bool inv, cudaStream_t s)
        : mem(sizeof(double) * (axis_pool_doubles(n[0]) + axis_pool_doubles(n[1]) + axis_pool_doubles(n[2]) +
                                (inv ? (size_t)n[0] * n[1] * n[2] : 0) + 64),
              s)
    {
        std::memset(&S, 0, sizeof(S));
        if (!mem.p) return;
        double* p = mem.as<double>();
        for (int d = 0; d < 3; d++) {
            S.n[d] = n[d];
            carve_axis(&S.ax[d], n[d], p);
            p += axis_pool_doubles(n[d]);
        }
        S.inv_diag = inv ? p : nullptr;
        const double* src[3] = {x, y, z};
        launch_level_tables(S, nullptr, src, 1, s);
        if (inv) launch_inv_diag(S, s);
    }
    bool ok() const { return mem.p != nullptr; }
};

}  // namespace

template <typename T>
int op_smooth_slab(const int n[3], const double* x, const double* y, const double* z, const T* u_in, T* u_out,
                   const T* b, int sweeps, int ns, int first, const int tile[3], void* stream)
{
    if (!op_grid_ok(n, x, y, z) || !u_in || !u_out || !b || !tile || u_in == u_out || sweeps < 1)
        return LASTO_ERR_INVALID_ARG;
    const SlabShape sh{tile[0], tile[1], tile[2], ns};
    if (!slab_shape_ok(sh, sizeof(T))) return LASTO_ERR_INVALID_ARG;
    init_device_constants();
    cudaStream_t s = (cudaStream_t)stream;
    OpLevel L(n, x, y, z, sizeof(T) == 8, s);
    if (!L.ok()) return LASTO_ERR_NO_MEMORY;
    const int full = sweeps / ns, rest = sweeps % ns, passes = full + (rest ? 1 : 0);
    Scratch tmp(passes > 1 ? sizeof(T) * (size_t)n[0] * n[1] * n[2] : 0, s);
    if (passes > 1 && !tmp.p) return LASTO_ERR_NO_MEMORY;
    const T* src = u_in;
    cudaError_t e = cudaSuccess;
    for (int m = 1; m <= passes && e == cudaSuccess; m++) {
        T* dst = ((passes - m) % 2 == 0) ? u_out : tmp.as<T>();   // the last pass lands in u_out
        SlabShape shm = sh;
        if (m == passes && rest) {   // the remainder pass (fewer sweeps) takes that kernel's own shape
            shm = slab_default_shape(rest, sizeof(T));
            shm.kz = sh.kz;
        }
        e = launch_rb_slab<T>(Arr<T>::view(L.S), src, dst, b, first & 1, 0, shm, s);
        src = dst;
    }
    return op_status(e);
}

extern "C" {

int lasto_op_sphere_params(const lasto_cluster* cl, double* q, double* rhoR, double* drhoR, double* coef, int* status,
                           void* stream)
{
    if (!cl || cl->n_atoms < 1 || !op_grid_ok(cl->n, cl->x, cl->y, cl->z)) return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    init_device_constants();
    Scratch rec(sizeof(double) * SPHERE_REC_DOUBLES * cl->n_atoms, s);
    if (!rec.p) return LASTO_ERR_NO_MEMORY;
    return op_status(launch_sphere_params(*cl, cl->x, cl->y, cl->z, rec.as<double>(), q, rhoR, drhoR, coef, status, s));
}

int lasto_op_deposit(const lasto_cluster* cl, int precision, double* b, int* owner, int* status, void* stream)
{
    if (!cl || !b || cl->n_atoms < 1 || !op_grid_ok(cl->n, cl->x, cl->y, cl->z)) return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    init_device_constants();
    Scratch rec(sizeof(double) * SPHERE_REC_DOUBLES * cl->n_atoms, s);
    if (!rec.p) return LASTO_ERR_NO_MEMORY;
    cudaError_t e = launch_sphere_params(*cl, cl->x, cl->y, cl->z, rec.as<double>(), nullptr, nullptr, nullptr,
                                         nullptr, status, s);
    if (e == cudaSuccess) e = launch_deposit(*cl, rec.as<double>(), precision, b, owner, nullptr, nullptr, status, s);
    return op_status(e);
}

int lasto_op_multipoles(const int n[3], const double* x, const double* y, const double* z, const double* b,
                        const double centre[3], double* Q, void* stream)
{
    if (!op_grid_ok(n, x, y, z) || !b || !centre || !Q) return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    init_device_constants();
    Scratch m(sizeof(double) * multipole_scratch_doubles(n), s);
    if (!m.p) return LASTO_ERR_NO_MEMORY;
    double* tabs = m.as<double>();
    double* rowm = tabs + 5 * ((size_t)n[0] + n[1] + n[2]);
    double* plane = rowm + 5 * (size_t)n[1] * n[2];
    return op_status(launch_multipoles(n, x, y, z, b, centre, tabs, rowm, plane, Q, s));
}

int lasto_op_boundary_fill(const int n[3], const double* x, const double* y, const double* z, const double centre[3],
                           const double* Q, double* u, void* stream)
{
    if (!op_grid_ok(n, x, y, z) || !centre || !Q || !u) return LASTO_ERR_INVALID_ARG;
    init_device_constants();
    return op_status(launch_boundary_fill(n, x, y, z, centre[0], centre[1], centre[2], Q, u, (cudaStream_t)stream));
}

int lasto_op_boundary_exact(const lasto_cluster* cl, double* u, void* stream)
{
    if (!cl || cl->n_atoms < 1 || !cl->pos || !cl->Z || !cl->R || !cl->slater_w || !cl->slater_zeta || !cl->c_lm ||
        !cl->x || !cl->y || !cl->z || !u)
        return LASTO_ERR_INVALID_ARG;
    for (int d = 0; d < 3; d++)
        if (cl->n[d] < 2) return LASTO_ERR_INVALID_ARG;
    init_device_constants();
    cudaStream_t s = (cudaStream_t)stream;
    Scratch M(sizeof(double) * 5 * (size_t)cl->n_atoms, s);
    if (!M.p) return LASTO_ERR_NO_MEMORY;
    return op_status(launch_boundary_exact(*cl, M.as<double>(), u, s));
}

int lasto_op_apply(const int n[3], const double* x, const double* y, const double* z, const double* u, double* Au,
                   void* stream)
{
    if (!op_grid_ok(n, x, y, z) || !u || !Au) return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    OpLevel L(n, x, y, z, false, s);
    if (!L.ok()) return LASTO_ERR_NO_MEMORY;
    return op_status(launch_apply<double>(L.S.view64(), u, Au, s));
}

int lasto_op_residual(const int n[3], const double* x, const double* y, const double* z, const double* u,
                      const double* b, double* r, void* stream)
{
    if (!op_grid_ok(n, x, y, z) || !u || !b || !r) return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    OpLevel L(n, x, y, z, false, s);
    if (!L.ok()) return LASTO_ERR_NO_MEMORY;
    return op_status(launch_residual<double>(L.S.view64(), u, b, r, s));
}

int lasto_op_smooth(const int n[3], const double* x, const double* y, const double* z, double* u, const double* b,
                    int sweeps, int threads, void* stream)
{
    if (!op_grid_ok(n, x, y, z) || !u || !b || sweeps < 0) return LASTO_ERR_INVALID_ARG;
    if (threads != 0 && (threads < 32 || threads > 512 || threads % 32)) return LASTO_ERR_INVALID_ARG;
    if (threads == 0 && n[0] > 1023) return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    OpLevel L(n, x, y, z, true, s);
    if (!L.ok()) return LASTO_ERR_NO_MEMORY;
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < sweeps && e == cudaSuccess; it++) {
        e = launch_rbgs<double>(L.S.view64(), u, b, 0, s, threads);
        if (e == cudaSuccess) e = launch_rbgs<double>(L.S.view64(), u, b, 1, s, threads);
    }
    return op_status(e);
}

int lasto_op_smooth_f32(const int n[3], const double* x, const double* y, const double* z, float* u, const float* b,
                        int sweeps, int threads, void* stream)
{
    if (!op_grid_ok(n, x, y, z) || !u || !b || sweeps < 0) return LASTO_ERR_INVALID_ARG;
    if (threads != 0 && (threads < 32 || threads > 512 || threads % 32)) return LASTO_ERR_INVALID_ARG;
    if (threads == 0 && n[0] > 1023) return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    OpLevel L(n, x, y, z, false, s);
    if (!L.ok()) return LASTO_ERR_NO_MEMORY;
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < sweeps && e == cudaSuccess; it++) {
        e = launch_rbgs<float>(L.S.view32(), u, b, 0, s, threads);
        if (e == cudaSuccess) e = launch_rbgs<float>(L.S.view32(), u, b, 1, s, threads);
    }
    return op_status(e);
}

int lasto_op_smooth_split_f32(const int n[3], const double* x, const double* y, const double* z, float* u,
                              const float* b, int sweeps, int threads, void* stream)
{
    if (!op_grid_ok(n, x, y, z) || !u || !b || sweeps < 0) return LASTO_ERR_INVALID_ARG;
    const bool staged = threads == RBGS_STAGED;
    if (threads != 0 && !staged && (threads < 32 || threads > 512 || threads % 32)) return LASTO_ERR_INVALID_ARG;
    if (threads == 0 && n[0] > 1023) return LASTO_ERR_INVALID_ARG;
    for (int d = 0; d < 3; d++)
        if (n[d] % 2 == 0) return LASTO_ERR_INVALID_ARG;   // the colour is the flat-index parity
    if (staged && (!split_stage_ok(n[0], n[1], n[2]) || ((uintptr_t)u & 15u) || ((uintptr_t)b & 15u)))
        return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    OpLevel L(n, x, y, z, false, s);
    if (!L.ok()) return LASTO_ERR_NO_MEMORY;
    LevelT<float> V = L.S.view32();
    set_split(V, true);
    // the staged kernel's bounded waits report into a device word read back at the end
    Scratch st(staged ? sizeof(int) : 0, s);
    if (staged && !st.p) return LASTO_ERR_NO_MEMORY;
    cudaError_t e = staged ? cudaMemsetAsync(st.p, 0, sizeof(int), s) : cudaSuccess;
    for (int it = 0; it < sweeps && e == cudaSuccess; it++) {
        e = launch_rbgs<float>(V, u, b, 0, s, threads, st.as<int>());
        if (e == cudaSuccess) e = launch_rbgs<float>(V, u, b, 1, s, threads, st.as<int>());
    }
    if (staged && e == cudaSuccess) {
        int flag = 0;
        e = cudaMemcpyAsync(&flag, st.p, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && flag) return flag;
    }
    return op_status(e);
}

int lasto_op_smooth_slab(const int n[3], const double* x, const double* y, const double* z, const double* u_in,
                         double* u_out, const double* b, int sweeps, int ns, int first, const int tile[3],
                         void* stream)
{
    return op_smooth_slab<double>(n, x, y, z, u_in, u_out, b, sweeps, ns, first, tile, stream);
}

int lasto_op_smooth_slab_f32(const int n[3], const double* x, const double* y, const double* z, const float* u_in,
                             float* u_out, const float* b, int sweeps, int ns, int first, const int tile[3],
                             void* stream)
{
    return op_smooth_slab<float>(n, x, y, z, u_in, u_out, b, sweeps, ns, first, tile, stream);
}

int lasto_op_smooth_wave_f32(const int n[3], const double* x, const double* y, const double* z, const float* u_in,
                             float* u_out, const float* b, int sweeps, int first, int tx, int ty, void* stream)
{
    if (!op_grid_ok(n, x, y, z) || !u_in || !u_out || !b || u_in == u_out || sweeps < 1) return LASTO_ERR_INVALID_ARG;
    const SlabShape sh{tx, ty, 8, 1};
    if (!wave_shape_ok(sh) || !wave_level_ok(n[0], n[1], n[2])) return LASTO_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(u_in) | reinterpret_cast<uintptr_t>(u_out) | reinterpret_cast<uintptr_t>(b)) & 15)
        return LASTO_ERR_INVALID_ARG;
    init_device_constants();
    cudaStream_t s = (cudaStream_t)stream;
    OpLevel L(n, x, y, z, false, s);
    if (!L.ok()) return LASTO_ERR_NO_MEMORY;
    Scratch tmp(sweeps > 1 ? sizeof(float) * (size_t)n[0] * n[1] * n[2] : 0, s);
    if (sweeps > 1 && !tmp.p) return LASTO_ERR_NO_MEMORY;
    const float* src = u_in;
    cudaError_t e = cudaSuccess;
    for (int m = 1; m <= sweeps && e == cudaSuccess; m++) {
        float* dst = ((sweeps - m) % 2 == 0) ? u_out : tmp.as<float>();   // the last pass lands in u_out
        e = launch_rb_wave(L.S.view32(), src, dst, b, first & 1, sh, s);
        src = dst;
    }
    return op_status(e);
}

int lasto_selftest_bounded_wait(double seconds, int* status, void* stream)
{
    if (!status || !(seconds > 0.0) || seconds > 60.0) return LASTO_ERR_INVALID_ARG;
    return op_status(launch_wait_selftest((unsigned long long)(seconds * 1e9), status, (cudaStream_t)stream));
}

int lasto_probe_fma(int precision, int blocks, int iters, void* out, void* stream)
{
    if ((precision != 0 && precision != 1) || blocks < 1 || iters < 1 || !out) return LASTO_ERR_INVALID_ARG;
    return op_status(launch_fma_probe(precision, blocks, iters, out, (cudaStream_t)stream));
}

int lasto_op_restrict(const int n[3], const double* x, const double* y, const double* z, const double* r, double* bc,
                      void* stream)
{
    if (!op_grid_ok(n, x, y, z) || !r || !bc || n[0] < 5 || n[1] < 5 || n[2] < 5) return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    OpLevel L(n, x, y, z, false, s);
    if (!L.ok()) return LASTO_ERR_NO_MEMORY;
    LevelT<double> C = L.S.view64();
    set_dims(C, (n[0] + 1) / 2, (n[1] + 1) / 2, (n[2] + 1) / 2);
    return op_status(launch_restrict<double>(L.S.view64(), C, r, bc, s));
}

int lasto_op_prolong_add(const int n[3], const double* x, const double* y, const double* z, const double* ec,
                         double* u, void* stream)
{
    if (!op_grid_ok(n, x, y, z) || !ec || !u || n[0] < 5 || n[1] < 5 || n[2] < 5) return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    OpLevel L(n, x, y, z, false, s);
    if (!L.ok()) return LASTO_ERR_NO_MEMORY;
    LevelT<double> C = L.S.view64();
    set_dims(C, (n[0] + 1) / 2, (n[1] + 1) / 2, (n[2] + 1) / 2);
    return op_status(launch_prolong_add<double>(L.S.view64(), C, ec, u, s));
}

int lasto_op_coarse_solve(const int n[3], const double* x, const double* y, const double* z, const double* b,
                          double* e, void* stream)
{
    if (!op_grid_ok(n, x, y, z) || !b || !e || n[0] > MAX_COARSE || n[1] > MAX_COARSE || n[2] > MAX_COARSE)
        return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    OpLevel L(n, x, y, z, false, s);
    Scratch eig(sizeof(CoarseEig), s);
    if (!L.ok() || !eig.p) return LASTO_ERR_NO_MEMORY;
    cudaError_t er = launch_coarse_eig(L.S, eig.as<CoarseEig>(), s);
    if (er == cudaSuccess) er = launch_coarse_apply<double>(L.S.view64(), eig.as<CoarseEig>(), b, e, false, s);
    return op_status(er);
}

int lasto_op_project(const int n[3], const double* x, const double* y, const double* z, const double* u, int n_atoms,
                     const double* pos, const double* R, int n_theta, int n_phi, double* vlm, int* status,
                     void* stream)
{
    if (!op_grid_ok(n, x, y, z) || !u || n_atoms < 0 || (n_atoms > 0 && (!pos || !R || !vlm)) || n_theta < 1 ||
        n_theta > 32 || n_phi < 1 || n_phi > 64)
        return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nq = n_theta * n_phi;
    std::vector<double> tab((size_t)nq * 28);
    host_quadrature(n_theta, n_phi, tab.data());
    Scratch q(sizeof(double) * tab.size(), s);
    if (!q.p) return LASTO_ERR_NO_MEMORY;
    cudaError_t e = cudaMemcpyAsync(q.p, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = launch_project(n, x, y, z, u, n_atoms, pos, R, q.as<double>(), nq, vlm, status, s);
    return op_status(e);
}

int lasto_op_sphere_density(const lasto_cluster* cl, int n_rad, double r_min, int n_theta, int n_phi, double* rho_lm,
                            int* status, void* stream)
{
    if (!cl || cl->n_atoms < 1 || !cl->pos || !cl->R || !cl->slater_w || !cl->slater_zeta || !cl->c_lm || !cl->x ||
        !cl->y || !cl->z || !rho_lm || n_rad < 4 || !(r_min > 0.0) || n_theta < 1 || n_theta > 32 || n_phi < 1 ||
        n_phi > 64)
        return LASTO_ERR_INVALID_ARG;
    for (int d = 0; d < 3; d++)
        if (cl->n[d] < 5) return LASTO_ERR_INVALID_ARG;
    init_device_constants();
    cudaStream_t s = (cudaStream_t)stream;
    const int nq = n_theta * n_phi;
    std::vector<double> tab((size_t)nq * 28);
    host_quadrature(n_theta, n_phi, tab.data());
    Scratch q(sizeof(double) * tab.size(), s);
    Scratch rec(sizeof(double) * SPHERE_REC_DOUBLES * (size_t)cl->n_atoms, s);
    if (!q.p || !rec.p) return LASTO_ERR_NO_MEMORY;
    cudaError_t e = cudaMemcpyAsync(q.p, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        e = launch_sphere_params(*cl, cl->x, cl->y, cl->z, rec.as<double>(), nullptr, nullptr, nullptr, nullptr,
                                 status, s);
    if (e == cudaSuccess)
        e = launch_sphere_density(cl->n_atoms, rec.as<double>(), cl->c_lm, q.as<double>(), nq, n_rad, r_min, rho_lm, s);
    return op_status(e);
}

int lasto_op_raw_deposit(const lasto_raw_cluster* cl, double* b, int* owner, int* status, void* stream)
{
    if (!cl || cl->n_atoms < 1 || !cl->pos || !cl->Z || !cl->R || !cl->x || !cl->y || !cl->z || !cl->density ||
        !cl->rho00 || cl->n_rad < 5 || !(cl->r_min > 0.0) || !b)
        return LASTO_ERR_INVALID_ARG;
    for (int d = 0; d < 3; d++)
        if (cl->n[d] < 5) return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch rec(sizeof(double) * RAW_REC * (size_t)cl->n_atoms, s);
    if (!rec.p) return LASTO_ERR_NO_MEMORY;
    const RawArgs ra = raw_args(*cl);
    cudaError_t e = launch_raw_sphere_params(ra, rec.as<double>(), status, s);
    if (e == cudaSuccess) e = launch_raw_deposit(ra, rec.as<double>(), b, owner, status, s);
    return op_status(e);
}

int lasto_op_inner_solve(int n_atoms, const double* R, const double* Z, int n_rad, double r_min, const double* rho_lm,
                         const double* v_R, double* v, void* stream)
{
    if (n_atoms < 1 || !R || !Z || n_rad < 4 || !(r_min > 0.0) || !rho_lm || !v_R || !v || rho_lm == v)
        return LASTO_ERR_INVALID_ARG;
    return op_status(launch_inner_solve(n_atoms, R, Z, n_rad, r_min, rho_lm, v_R, v, (cudaStream_t)stream));
}

int lasto_op_interstitial_hs(const int n[3], const double* x, const double* y, const double* z, int n_atoms,
                             const double* pos, const double* R, int nb, const int* bn, const int* bl, const double* bz,
                             const double* V, double* S, double* H, int mode, lasto_hs_stats* stats,
                             void* stream)
{
    if (!n || !x || !y || !z || n_atoms < 1 || !pos || !R || !V || !S || !H || S == H) return LASTO_ERR_INVALID_ARG;
    for (int d = 0; d < 3; d++)
        if (n[d] < 2) return LASTO_ERR_INVALID_ARG;
    if ((size_t)n[0] * n[1] * n[2] >= ((size_t)1 << 31)) return LASTO_ERR_INVALID_ARG;
    int per = 0;
    if (hs_basis_check(nb, bn, bl, bz, &per) != LASTO_OK) return LASTO_ERR_INVALID_ARG;
    if ((size_t)n_atoms * per > 65536) return LASTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch w(hs_scratch_bytes(n, n_atoms * per, n_atoms), s);
    if (!w.p) return LASTO_ERR_NO_MEMORY;
    return launch_interstitial_hs(n, x, y, z, n_atoms, pos, R, nb, bn, bl, bz, V, S, H, w.p, mode, stats, s);
}

}  // extern "C"
