// Internal declarations of the sm_103a LASTO interstitial Poisson library.
// Shared only among the library's own .cu files.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/lasto_poisson.h"

namespace lasto {

constexpr int NLM = 25;
constexpr int MAX_LEVELS = 10;
constexpr int MAX_COARSE = 9;        // nodes per axis on the coarsest level
constexpr int MAX_QUAD = 2048;       // n_theta * n_phi
constexpr int RED_THREADS = 256;     // block size of reducing kernels
constexpr double PI = 3.141592653589793238462643383279502884;

// ---------------------------------------------------------------- errors
struct Err {
    int code = LASTO_OK;
    std::string msg;
};
int set_cuda_error(Err* e, cudaError_t c, const char* what);
#define LASTO_TRY(err, call)                                              \
    do {                                                                  \
        cudaError_t c_ = (call);                                          \
        if (c_ != cudaSuccess) return ::lasto::set_cuda_error(err, c_, #call); \
    } while (0)

// Status of a single-operation entry point from the CUDA error of its launches.
inline int op_status(cudaError_t e) { return e == cudaSuccess ? LASTO_OK : LASTO_ERR_CUDA; }

// The grid conditions every single-operation entry point checks: three axis arrays, an odd
// number (>= 3) of nodes per axis, and fewer than 2^31 nodes (kernels index with 31 bits).
inline bool op_grid_ok(const int n[3], const double* x, const double* y, const double* z)
{
    if (!n || !x || !y || !z) return false;
    for (int d = 0; d < 3; d++)
        if (n[d] < 3 || n[d] % 2 == 0) return false;
    return (size_t)n[0] * n[1] * n[2] < (size_t(1) << 31);
}

// ---------------------------------------------------------------- spherical harmonics
// Real solid harmonics r^l y_lm as sums of monomials x^a y^b z^c (a+b+c = l <= 4).
struct Mono {
    int lm;
    int a, b, c;
    double coef;
};
constexpr int N_MONO_TERMS = 56;
void host_monomials(Mono* out);      // the 56 terms, coefficients in FP64
void host_solid_harmonics(double x, double y, double z, double* S);

__host__ __device__ __forceinline__ int l_of_lm(int lm) { return lm >= 16 ? 4 : lm >= 9 ? 3 : lm >= 4 ? 2 : lm >= 1 ? 1 : 0; }

// ---------------------------------------------------------------- FP32 point update
// u = acc / (-dsum) of a red-black FP32 update as acc times the hardware's approximate
// reciprocal (rcp.approx.ftz.f32, relative error below 2^-23 for the diagonal's range, one
// instruction): the same expression in every FP32 smoother variant, so they stay bitwise equal.
// The correctly rounded reciprocal costs a Newton step and a special-case branch per node, about
// 6 % of the row-per-warp half sweep's time; a smoother's update needs no last-bit rounding.
__device__ __forceinline__ float rb_point32(float acc, float dsum)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-dsum));
    return acc * r;
}

// ---------------------------------------------------------------- block reductions
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* smem)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) smem[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < NT / 32) ? smem[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;  // valid in thread 0
}

// ---------------------------------------------------------------- levels
// Per-axis tables of one level.  Coordinates and every coefficient derive from the
// node coordinates of the level (the coarse level keeps every other fine node).
template <typename T>
struct AxisT {
    const double* c;   // coordinates [n]
    const T* cm;       // 2/((h- + h+) h-)  (minus neighbour) [n], 0 at the ends
    const T* cp;       // 2/((h- + h+) h+)  (plus neighbour)
    const T* dg;       // cm + cp
    const T* dual;     // dual-cell length
    const T* pl;       // prolongation weight of coarse node (f-1)/2 at odd fine f (1 at even f)
    const T* pr;       // weight of coarse node (f+1)/2 at odd f (0 at even f)
    const T* rw;       // restriction weights of coarse node I [nc][3] (fine 2I-1, 2I, 2I+1)
    int n;
};

// Division of a node index by an invariant divisor as a multiply-high and a shift: with
// 2^(l-1) < d <= 2^l and m = ceil(2^(31+l) / d) (which fits in 32 bits), floor(n / d) =
// floor(m n / 2^(31+l)) for every 0 <= n < 2^31 (Granlund and Montgomery, "Division by
// invariant integers using multiplication", 1994, Theorem 4.2 with N = 31).  Node indices stay
// below 2^31 (checked where grids are accepted).
struct DivMagic {
    unsigned m;
    int s;   // l - 1
};

inline DivMagic div_magic(unsigned d)
{
    int l = 0;
    while ((1ull << l) < d) l++;
    DivMagic r;
    r.m = (unsigned)(((1ull << (31 + l)) + d - 1) / d);
    r.s = l - 1;
    return r;
}

__device__ __forceinline__ unsigned div_by(unsigned n, DivMagic q)
{
    return __umulhi(n, q.m) >> q.s;
}

// Storage order of a level's node arrays.  Natural: node P (flat index, x fastest) at P.
// Colour-split: the even flat indices (red, i+j+k even, as every axis has an odd node count)
// first, in order, then the odd ones: node P at (P >> 1) + (P & 1) H, H = ceil(N / 2).  Every
// neighbour of a node has the other colour, so a half sweep over split storage reads only the
// other half and its own right-hand side and writes only its own half, all with unit stride,
// where natural storage moves every sector of both colours in each half sweep.
template <typename T>
struct LevelT {
    AxisT<T> ax[3];
    const T* inv_diag;  // [N] or nullptr (FP32 smoother computes the diagonal)
    int nx, ny, nz;
    DivMagic dvx, dvxy;  // division by nx and by nx * ny (set_dims)
    unsigned lsh;        // 0: natural storage; 1: colour-split storage
    unsigned H;          // colour-split: offset of the odd half, ceil(N / 2); natural: 0
    __host__ __device__ size_t N() const { return (size_t)nx * ny * nz; }
};

// The only way dimensions are set: keeps the division constants in step (every axis >= 3 nodes);
// natural storage.
template <typename T>
inline void set_dims(LevelT<T>& v, int nx, int ny, int nz)
{
    v.nx = nx;
    v.ny = ny;
    v.nz = nz;
    v.dvx = div_magic((unsigned)nx);
    v.dvxy = div_magic((unsigned)nx * (unsigned)ny);
    v.lsh = 0;
    v.H = 0;
}

template <typename T>
inline void set_split(LevelT<T>& v, bool split)
{
    v.lsh = split ? 1u : 0u;
    v.H = split ? (unsigned)((v.N() + 1) / 2) : 0u;
}

// storage position of flat node P (nodes < 2^31)
template <typename T>
__host__ __device__ __forceinline__ unsigned at(const LevelT<T>& L, unsigned P)
{
    return (P >> L.lsh) + (P & L.lsh) * L.H;
}

// Raw (writable) per-axis storage of one level in one pool.
struct AxisStore {
    double* c;
    double *cm, *cp, *dg, *dual, *pl, *pr, *rw;
    float *cm32, *cp32, *dg32, *dual32, *pl32, *pr32, *rw32;
    int n;
};

struct LevelStore {
    AxisStore ax[3];
    int n[3];
    double* inv_diag;   // FP64 [N]
    double *u, *b, *r;  // FP64 work arrays (level 0: u unused by the preconditioner)
    double* u2;         // FP64 partner of the fused smoother passes (FP32 levels use r32)
    float *u32, *b32, *r32;
    bool split32 = false;   // the FP32 arrays in colour-split storage (view32 says so)
    size_t N() const { return (size_t)n[0] * n[1] * n[2]; }
    LevelT<double> view64() const;
    LevelT<float> view32() const;
};

// Exact coarse solve by fast diagonalisation of the three 1-D operators.
struct CoarseEig {
    double F[3][(MAX_COARSE - 2) * (MAX_COARSE - 2)];  // forward  [p][i] = Q[i][p] sqrt(V_i)
    double B[3][(MAX_COARSE - 2) * (MAX_COARSE - 2)];  // backward [i][p] = Q[i][p] / sqrt(V_i)
    double lam[3][MAX_COARSE - 2];
    int m[3];
    int ok[3];
};

int num_levels(const int n[3], int* coarse_n = nullptr);
size_t axis_pool_doubles(int n);     // doubles needed by one AxisStore of n nodes
void carve_axis(AxisStore* a, int n, double* pool);

// ---------------------------------------------------------------- kernel launchers
// mesh.cu
cudaError_t launch_mesh_axis(int n, double c, double L, double h_min, double h_max, double p_max, double* x,
                             double* info, cudaStream_t s);
cudaError_t launch_level_tables(const LevelStore& fine, const LevelStore* coarse, const double* src_coords[3],
                                int src_stride, cudaStream_t s);
cudaError_t launch_inv_diag(const LevelStore& L, cudaStream_t s);
cudaError_t launch_coarse_eig(const LevelStore& L, CoarseEig* eig, cudaStream_t s);

// mg.cu
// nt: threads per block of the flat kernels (32 .. 512), 0 for one warp (colour-split storage)
// or one block (natural) per row, RBGS_STAGED for the plane-staged kernel of stage.cu
// (colour-split FP32 only); status (may be null) receives LASTO_ERR_TIMEOUT from its bounded waits
constexpr int RBGS_STAGED = 1;
template <typename T>
cudaError_t launch_rbgs(const LevelT<T>& L, T* u, const T* b, int colour, cudaStream_t s, int nt = 256,
                        int* status = nullptr);
// the first red FP32 half sweep from u = 0 (either storage order; faces of u already zero)
cudaError_t launch_first_red32(const LevelT<float>& L, float* u, const float* b, cudaStream_t s);
// stage.cu
cudaError_t launch_split_stage(const LevelT<float>& L, float* u, const float* b, int colour, int* status, cudaStream_t s);
cudaError_t launch_split_stage_resid(const LevelT<float>& L, const float* u, const float* b, float* r, int* status,
                                     cudaStream_t s);
cudaError_t launch_split_stage_first_red(const LevelT<float>& L, float* u, const float* b, int* status, cudaStream_t s);
cudaError_t launch_prolong_stage(const LevelT<float>& F, const LevelT<float>& C, const float* ec, float* u, int* status,
                                 cudaStream_t s);
bool split_stage_ok(int nx, int ny, int nz);
void init_stage_attributes();
template <typename T>
cudaError_t launch_residual(const LevelT<T>& L, const T* u, const T* b, T* r, cudaStream_t s);
template <typename T>
cudaError_t launch_apply(const LevelT<T>& L, const T* u, T* Au, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict(const LevelT<T>& fine, const LevelT<T>& coarse, const T* r, T* bc, cudaStream_t s);
template <typename T>
cudaError_t launch_prolong_add(const LevelT<T>& fine, const LevelT<T>& coarse, const T* ec, T* u, cudaStream_t s,
                               int* status = nullptr);
template <typename T>
cudaError_t launch_coarse_apply(const LevelT<T>& L, const CoarseEig* eig, const T* b, T* e, bool add, cudaStream_t s);

// red_only (FP32): the fine iterate's last half sweep was black, so only the red residuals are
// formed (the black ones are zero).  scratch (optional, FP32, a free fine-level array, 16-byte
// aligned): over colour-split storage on a grid the staged kernels take, the red residuals are
// formed once into it by the plane-staged kernel and then restricted (status: its bounded waits)
template <typename T>
cudaError_t launch_resid_restrict(const LevelT<T>& fine, const LevelT<T>& coarse, const T* u, const T* b, T* bc, T* uc,
                                  bool red_only, cudaStream_t s, T* scratch = nullptr, int* status = nullptr);

// slab.cu: fused red-black smoother.  One pass = ns full sweeps (colour `first`, then the
// other), u_in -> u_out (distinct arrays; every node of u_out written).  A CTA owns a
// tx x ty tile of the (x, y) plane and kz planes of z.
struct SlabShape {
    int tx, ty, kz, ns;
};
constexpr size_t SLAB_MAX_SMEM = 200 * 1024;
size_t slab_smem_bytes(const SlabShape& sh, size_t elem);
bool slab_shape_ok(const SlabShape& sh, size_t elem);
SlabShape slab_default_shape(int ns, size_t elem);   // a valid shape for ns sweeps per pass
void init_slab_attributes();   // shared-memory opt-in; call outside capture
// zero_in != 0: u_in is taken as zero everywhere (it is not read)
template <typename T>
cudaError_t launch_rb_slab(const LevelT<T>& L, const T* uin, T* uout, const T* b, int first, int zero_in,
                           const SlabShape& sh, cudaStream_t s);

// wave.cu: fused red-black sweep as a z wavefront over row chunks staged in shared memory
// (FP32).  One pass = one full sweep (colour `first`, then the other), u_in -> u_out
// (distinct, 16-byte aligned; every node of u_out written, faces copied).  Shape: tx (16..60)
// columns and ty (8, 12 or 16) rows per tile, kz = 8 (the ring of staged planes); levels of at
// least 69 nodes per row.
bool wave_shape_ok(const SlabShape& sh);
bool wave_level_ok(int nx, int ny, int nz);
void init_wave_attributes();   // shared-memory opt-in; call outside capture
cudaError_t launch_rb_wave(const LevelT<float>& L, const float* uin, float* uout, const float* b, int first,
                           const SlabShape& sh, cudaStream_t s);
// probe.cu: one thread waits on an mbarrier nothing arrives at, for limit_ns, then raises TIMEOUT
cudaError_t launch_wait_selftest(unsigned long long limit_ns, int* status, cudaStream_t s);

// probe.cu: arithmetic throughput probes (FMA chains on every SM)
cudaError_t launch_fma_probe(int precision, int blocks, int iters, void* out, cudaStream_t s);

// Levels lb..L-1 of a V-cycle in one thread block (u[0] = 0 on entry).
constexpr int BOTTOM_MAX_LEVELS = 4;
constexpr size_t BOTTOM_MAX_NODES = 5000;    // the top bottom level has at most this many nodes (17^3)
template <typename T>
struct BottomArgs {
    LevelT<T> lv[BOTTOM_MAX_LEVELS];
    T* u[BOTTOM_MAX_LEVELS];
    T* b[BOTTOM_MAX_LEVELS];
    const CoarseEig* eig;
    int nlev, nu1, nu2, sym;
};
template <typename T>
cudaError_t launch_bottom(const BottomArgs<T>& a, cudaStream_t s);
void init_mg_attributes();   // shared-memory opt-in of the bottom kernel; call outside capture

// reductions / CG (mg.cu).  A reducing kernel sums one quantity over the grid and its last
// block applies the scalar step `op` (enum FinOp) to the control block.
struct Ctl;
struct Red {
    double* part;            // one partial per block (at most 1216 blocks)
    unsigned int* counter;   // zero between launches
    Ctl* ctl;
    int op;
    cudaGraphConditionalHandle cond;
    int use_cond;
};
int reduce_blocks(const LevelT<double>& L);
cudaError_t launch_bnorm(const LevelT<double>& L, const double* u, const double* b, const Red& red, cudaStream_t s);
cudaError_t launch_resid_norm(const LevelT<double>& L, const double* u, const double* b, double* r, float* r32,
                              unsigned h32, const Red& red, cudaStream_t s);
cudaError_t launch_apply_dot(const LevelT<double>& L, const double* p, double* q, const Red& red, cudaStream_t s);
cudaError_t launch_update_ur(const LevelT<double>& L, const Ctl* ctl, const double* p, const double* q, double* u,
                             double* r, const Red& red, cudaStream_t s);
cudaError_t launch_dot_rz(const LevelT<double>& L, const double* r, const double* z, const Red& red, cudaStream_t s);
cudaError_t launch_update_p(const LevelT<double>& L, const Ctl* ctl, const double* z, double* p, cudaStream_t s);
cudaError_t launch_apply_dot32(const LevelT<float>& L, const float* p, float* q, const Red& red, cudaStream_t s,
                               int* status = nullptr);
cudaError_t launch_update_er32(const LevelT<float>& L, const Ctl* ctl, const float* p, const float* q, float* e,
                               float* r, const Red& red, cudaStream_t s);
cudaError_t launch_dot32(const LevelT<float>& L, const float* r, const float* z, const Red& red, cudaStream_t s);
cudaError_t launch_update_p32(const LevelT<float>& L, const Ctl* ctl, const float* z, float* p, cudaStream_t s);
// (e in colour-split storage when h32 = ceil(N / 2) is nonzero)
cudaError_t launch_add_correction(size_t N, double* u, float* e, unsigned h32, cudaStream_t s);
cudaError_t launch_to_f32(const double* a, float* b, size_t n, cudaStream_t s);

// density.cu
void init_device_constants();   // constant tables and kernel attributes; call outside stream capture
constexpr int SPHERE_REC_DOUBLES = 48;
cudaError_t launch_sphere_params(const lasto_cluster& cl, const double* ax0, const double* ax1, const double* ax2,
                                 double* rec, double* q, double* rhoR, double* drhoR, double* coef, int* status,
                                 cudaStream_t s);
cudaError_t launch_deposit(const lasto_cluster& cl, const double* rec, int precision, double* b, int* owner,
                           const double* xm_tab, double* row_mom, int* status, cudaStream_t s);
size_t multipole_scratch_doubles(const int n[3]);
cudaError_t launch_multipoles(const int n[3], const double* x, const double* y, const double* z, const double* b,
                              const double centre[3], double* tabs, double* row_mom, double* plane, double* Q,
                              cudaStream_t s);
cudaError_t launch_boundary_exact(const lasto_cluster& cl, double* M, double* u, cudaStream_t s);   // M: 5 n_atoms scratch
cudaError_t launch_boundary_fill(const int n[3], const double* x, const double* y, const double* z, double cx,
                                 double cy, double cz, const double* Q, double* u, cudaStream_t s);

// raw.cu: the raw-density entry point (grid density + each sphere's rho_00 table)
struct RawArgs {
    int na;
    const double *pos, *Z, *R;
    int n[3];
    const double* ax[3];
    const double* ne;      // [N] electron density at the nodes
    int n_rad;
    double r_min;
    const double* rho00;   // [na][n_rad]
};
constexpr int RAW_REC = 8;   // x y z R a b c h per sphere
cudaError_t launch_raw_sphere_params(const RawArgs& a, double* rec, int* status, cudaStream_t s);
cudaError_t launch_raw_deposit(const RawArgs& a, const double* rec, double* b, int* owner, int* status, cudaStream_t s);

// inner.cu: inside the spheres (Eq. 3.4-3.7)
cudaError_t launch_sphere_density(int na, const double* rec, const double* clm, const double* quad, int nq,
                                  int n_rad, double r_min, double* out, cudaStream_t s);
cudaError_t launch_inner_solve(int na, const double* R, const double* Z, int n_rad, double r_min,
                               const double* rho_lm, const double* vR, double* v, cudaStream_t s);

// hs.cu: interstitial H and S (Eq. 3.11-3.14)
int hs_basis_check(int nb, const int* bn, const int* bl, const double* bz, int* per_out);
size_t hs_scratch_bytes(const int n[3], int M, int na);
int launch_interstitial_hs(const int n[3], const double* x, const double* y, const double* z, int na,
                           const double* pos, const double* R, int nb, const int* bn, const int* bl,
                           const double* bz, const double* V, double* S, double* H, void* scratch, int mode,
                           lasto_hs_stats* stats, cudaStream_t s);

// guess.cu: the learned initial guess (a 3-D U-Net on a 33^3 subgrid)
constexpr int GUESS_N = 33;
struct GuessNet;
size_t guess_param_count();
int guess_net_create(const float* params, size_t n_params, const double scales[4], int nbmax, GuessNet** out,
                     cudaStream_t s);
void guess_net_free(GuessNet* g);
int guess_net_forward(GuessNet* g, int nb, cudaStream_t s);
float* guess_net_features(GuessNet* g, int k);          // FP32 [33^3][16] input of grid k
const float* guess_net_prediction(GuessNet* g, int k);  // FP32 [33^3][16], channel 0 = prediction
int guess_net_capacity(const GuessNet* g);
const float* guess_net_scales(const GuessNet* g);       // s0, s1, h_ref, out
// nn.cu: convolution with an optional FP32 scratch for tap-group partial sums (small grids)
int conv_fwd(int nb, const int dims[3], int cin, int cout, const void* x, const void* w, const float* bias, int relu,
             float* y32, int ldy32, int off32, void* y16, int ldy16, int off16, float* scratch,
             size_t scratch_floats, void* stream);
// conv_tc.cu: the same convolution on tcgen05 tensor cores; weights packed once per set
cudaError_t launch_pack_weights(int cin, int cout, const void* w, void* wpk, cudaStream_t s);
int conv_fwd_tc(int nb, const int dims[3], int cin, int cout, const void* x, const void* wpk, const float* bias,
                int relu, float* y32, int ldy32, int off32, void* y16, int ldy16, int off16, float* scratch,
                size_t scratch_floats, int* err, void* stream);
// dw (FP32 [27][cin][cout]) += weight gradient on the tensor cores (FP32 atomics)
int conv_wgrad_tc(int nb, const int dims[3], int cin, int cout, const void* x, const void* dy16, float* dw,
                  int* err, void* stream);
cudaError_t launch_axis_stride(const double* src, int m, int n, double* dst, cudaStream_t s);
cudaError_t launch_resample(const int na[3], const double* ax, const double* ay, const double* az, const double* src,
                            const int nb[3], const double* bx, const double* by, const double* bz, double* dst,
                            int interior_only, cudaStream_t s);

// project.cu
void host_quadrature(int n_theta, int n_phi, double* table /* [nq][28]: unit xyz, w*S_lm */);
cudaError_t launch_project(const int n[3], const double* x, const double* y, const double* z, const double* u,
                           int n_atoms, const double* pos, const double* R, const double* quad, int nq,
                           double* vlm, int* status, cudaStream_t s);

// ---------------------------------------------------------------- lockstep batches (mg.cu)
// Clusters whose grids have the same shape advance together: each kernel of the FP32 cycle and
// of the CG / defect-correction steps is launched once for all members (blockIdx.y = member,
// blockIdx.x as in the single-cluster launch), and a member whose loop has ended returns at the
// top of every block.  `mode` picks the member's flag: BAT_INNER runs while its inner CG goes on
// (Ctl::go_in), BAT_OUTER while its defect correction is not done.  Each member keeps its own
// control block and reduction partials, so its arithmetic and sums are those of a
// single-cluster launch.
enum BatMode { BAT_INNER = 1, BAT_OUTER = 2 };

struct BatLevel {            // one member's FP32 level l and l + 1
    LevelT<float> V, VC;
    float *u, *b, *uc, *bc;
    const Ctl* ctl;
};
struct BatVec {              // one member's finest-level vectors, partials and control block
    LevelT<float> V32;
    LevelT<double> V64;
    float *u32, *b32, *e32, *p32, *q32;
    double *u, *b, *r;
    double* part;
    unsigned int* counter;
    Ctl* ctl;
    int* status;             // the member's solve status (bounded waits of the staged kernels)
};
struct BatBottom {           // one member's one-block bottom levels
    BottomArgs<float> a;
    const Ctl* ctl;
};

// A group's member arguments, passed by value as a kernel parameter (constant bank; member =
// blockIdx.y), at most BAT_MAX members.
constexpr int BAT_MAX = 16;
template <typename A>
struct BatPack {
    A m[BAT_MAX];
};

// In-place FP32 half sweep of colour `colour` on every member's level (V0: the shared shape):
// the flat-index kernel (nt threads) in natural storage, one warp per row in colour-split storage.
cudaError_t launch_rbgs_bat(const LevelT<float>& V0, const BatPack<BatLevel>& m, int nm, int colour, int nt,
                            cudaStream_t s);
cudaError_t launch_resid_restrict_bat(const LevelT<float>& F0, const LevelT<float>& C0, const BatPack<BatLevel>& m,
                                      int nm, bool red_only, cudaStream_t s);
cudaError_t launch_prolong_add_bat(const LevelT<float>& F0, const LevelT<float>& C0, const BatPack<BatLevel>& m,
                                   int nm, cudaStream_t s);
cudaError_t launch_bottom_bat(const BottomArgs<float>& a0, const BatBottom* m, int nm, cudaStream_t s);
// finest-level steps; `op` the reduction's scalar step (FinOp)
cudaError_t launch_zero_bat(const BatPack<BatVec>& m, int nm, size_t n, int which, int mode, cudaStream_t s);
cudaError_t launch_dot32_bat(const LevelT<float>& V0, const BatPack<BatVec>& m, int nm, int with_z, int op, int mode,
                             cudaStream_t s);
cudaError_t launch_update_p32_bat(const LevelT<float>& V0, const BatPack<BatVec>& m, int nm, cudaStream_t s);
cudaError_t launch_apply_dot32_bat(const LevelT<float>& V0, const BatPack<BatVec>& m, int nm, cudaStream_t s);
cudaError_t launch_update_er32_bat(const LevelT<float>& V0, const BatPack<BatVec>& m, int nm, cudaStream_t s);
cudaError_t launch_outer_bat(const LevelT<double>& V0, const BatPack<BatVec>& m, int nm, unsigned h32,
                             cudaStream_t s);
// the loop condition of a batch: 1 while any member's flag (mode) is set
cudaError_t launch_any_bat(Ctl* const* ctls, int nm, int mode, cudaGraphConditionalHandle cond, cudaStream_t s);

}  // namespace lasto
