// Right-hand side of the interstitial Poisson problem: per-sphere pseudo-density,
// deposit on the mesh, boundary multipoles and Dirichlet face values.
//
// Section 1 of the paper: the rapidly varying density inside each sphere is replaced
// by a smooth pseudo-density with the same multipole moments (nucleus included); only
// the monopole is replaced, the nonspherical terms go on the grid as they are.
// Section 3 (constraints beside Eq. 3.2-3.3): same charge inside the sphere, same
// value and slope at R.  Reading of the shape: rho_tilde = a + b r^2 + c r^4.
//
// GPU formulation.  With the same three Slater exponents on every atom, the spherical
// average of the neighbours' Slater terms about sphere i factorises into
//   N_i(r) = sum_k [ 2 A_ik sinh(zeta_k r)/r - 2 B_ik cosh(zeta_k r) ],
//   A_ik = sum_{j != i} W_jk e^{-zeta_k D_ij} (1 + zeta_k D_ij) / (2 D_ij zeta_k^2),
//   B_ik = sum_{j != i} W_jk e^{-zeta_k D_ij} / (2 D_ij zeta_k),
// (W = w zeta^3 / 8 pi), so a node inside sphere i costs three exponentials instead
// of one average per neighbour, and the sphere charge integrals are closed forms.
// Inside sphere i the deposit evaluates n_e - rho0_i + rho_tilde_i as
//   (neighbours' Slater terms at the node) - N_i(r) + rho_ns,i(x) + rho_tilde_i(r),
// the atom's own spherical terms cancelling exactly rather than numerically.
#include <cmath>

#include "df.cuh"
#include <mutex>

#include "internal.cuh"

namespace lasto {

// ---------------------------------------------------------------- harmonics table
static __constant__ Mono c_mono[N_MONO_TERMS];

// double-float copies for the FP32-pair deposit
struct MonoF {
    int lm, a, b, c;
    float h, l;
};
static __constant__ MonoF c_mono_f[N_MONO_TERMS];
static __constant__ float c_exp_h[64], c_exp_l[64];   // 2^(-j/64) as double-floats

void host_monomials(Mono* o)
{
    const double pi = PI;
    const double c0 = 0.5 / std::sqrt(pi), c1 = std::sqrt(3.0 / (4 * pi));
    const double c2a = 0.5 * std::sqrt(15 / pi), c2b = 0.25 * std::sqrt(5 / pi), c2c = 0.25 * std::sqrt(15 / pi);
    const double c3a = 0.25 * std::sqrt(35 / (2 * pi)), c3b = 0.5 * std::sqrt(105 / pi), c3c = 0.25 * std::sqrt(21 / (2 * pi));
    const double c3d = 0.25 * std::sqrt(7 / pi), c3e = 0.25 * std::sqrt(105 / pi);
    const double c4a = 0.75 * std::sqrt(35 / pi), c4b = 0.75 * std::sqrt(35 / (2 * pi)), c4c = 0.75 * std::sqrt(5 / pi);
    const double c4d = 0.75 * std::sqrt(5 / (2 * pi)), c4e = (3.0 / 16) / std::sqrt(pi), c4f = 0.375 * std::sqrt(5 / pi);
    const double c4g = (3.0 / 16) * std::sqrt(35 / pi);
    const Mono t[N_MONO_TERMS] = {
        {0, 0, 0, 0, c0},
        {1, 0, 1, 0, c1}, {2, 0, 0, 1, c1}, {3, 1, 0, 0, c1},
        {4, 1, 1, 0, c2a}, {5, 0, 1, 1, c2a},
        {6, 0, 0, 2, 2 * c2b}, {6, 2, 0, 0, -c2b}, {6, 0, 2, 0, -c2b},
        {7, 1, 0, 1, c2a}, {8, 2, 0, 0, c2c}, {8, 0, 2, 0, -c2c},
        {9, 2, 1, 0, 3 * c3a}, {9, 0, 3, 0, -c3a},
        {10, 1, 1, 1, c3b},
        {11, 0, 1, 2, 4 * c3c}, {11, 2, 1, 0, -c3c}, {11, 0, 3, 0, -c3c},
        {12, 0, 0, 3, 2 * c3d}, {12, 2, 0, 1, -3 * c3d}, {12, 0, 2, 1, -3 * c3d},
        {13, 1, 0, 2, 4 * c3c}, {13, 3, 0, 0, -c3c}, {13, 1, 2, 0, -c3c},
        {14, 2, 0, 1, c3e}, {14, 0, 2, 1, -c3e},
        {15, 3, 0, 0, c3a}, {15, 1, 2, 0, -3 * c3a},
        {16, 3, 1, 0, c4a}, {16, 1, 3, 0, -c4a},
        {17, 2, 1, 1, 3 * c4b}, {17, 0, 3, 1, -c4b},
        {18, 1, 1, 2, 6 * c4c}, {18, 3, 1, 0, -c4c}, {18, 1, 3, 0, -c4c},
        {19, 0, 1, 3, 4 * c4d}, {19, 2, 1, 1, -3 * c4d}, {19, 0, 3, 1, -3 * c4d},
        {20, 0, 0, 4, 8 * c4e}, {20, 4, 0, 0, 3 * c4e}, {20, 0, 4, 0, 3 * c4e},
        {20, 2, 2, 0, 6 * c4e}, {20, 2, 0, 2, -24 * c4e}, {20, 0, 2, 2, -24 * c4e},
        {21, 1, 0, 3, 4 * c4d}, {21, 3, 0, 1, -3 * c4d}, {21, 1, 2, 1, -3 * c4d},
        {22, 2, 0, 2, 6 * c4f}, {22, 0, 2, 2, -6 * c4f}, {22, 4, 0, 0, -c4f}, {22, 0, 4, 0, c4f},
        {23, 3, 0, 1, c4b}, {23, 1, 2, 1, -3 * c4b},
        {24, 4, 0, 0, c4g}, {24, 2, 2, 0, -6 * c4g}, {24, 0, 4, 0, c4g},
    };
    for (int i = 0; i < N_MONO_TERMS; i++) o[i] = t[i];
}

void host_solid_harmonics(double x, double y, double z, double* S)
{
    Mono t[N_MONO_TERMS];
    host_monomials(t);
    double px[5] = {1, x, x * x, x * x * x, x * x * x * x}, py[5] = {1, y, y * y, y * y * y, y * y * y * y},
           pz[5] = {1, z, z * z, z * z * z, z * z * z * z};
    for (int q = 0; q < NLM; q++) S[q] = 0.0;
    for (int i = 0; i < N_MONO_TERMS; i++) S[t[i].lm] += t[i].coef * px[t[i].a] * py[t[i].b] * pz[t[i].c];
}

// Constant tables are per device: each device gets its own upload, once, with that device
// current (a flag per device, so alternating devices uploads nothing again).
constexpr int MAX_DEVICES = 64;
static bool g_mono_uploaded[MAX_DEVICES] = {};
static bool g_constants_done[MAX_DEVICES] = {};
static std::mutex g_constants_mutex;

static cudaError_t ensure_monomials()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_constants_mutex);
    if (g_mono_uploaded[dev]) return cudaSuccess;
    Mono t[N_MONO_TERMS];
    host_monomials(t);
    e = cudaMemcpyToSymbol(c_mono, t, sizeof(t));
    if (e != cudaSuccess) return e;
    MonoF tf[N_MONO_TERMS];
    for (int i = 0; i < N_MONO_TERMS; i++) {
        tf[i].lm = t[i].lm;
        tf[i].a = t[i].a;
        tf[i].b = t[i].b;
        tf[i].c = t[i].c;
        tf[i].h = (float)t[i].coef;
        tf[i].l = (float)(t[i].coef - (double)tf[i].h);
    }
    e = cudaMemcpyToSymbol(c_mono_f, tf, sizeof(tf));
    if (e != cudaSuccess) return e;
    float eh[64], el[64];
    for (int j = 0; j < 64; j++) {
        const double v = std::exp2(-j / 64.0);
        eh[j] = (float)v;
        el[j] = (float)(v - (double)eh[j]);
    }
    e = cudaMemcpyToSymbol(c_exp_h, eh, sizeof(eh));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_exp_l, el, sizeof(el));
    if (e == cudaSuccess) g_mono_uploaded[dev] = true;
    return e;
}

__device__ __forceinline__ void solid_harmonics(double x, double y, double z, double* S)
{
    double px[5], py[5], pz[5];
    px[0] = py[0] = pz[0] = 1.0;
#pragma unroll
    for (int p = 1; p < 5; p++) {
        px[p] = px[p - 1] * x;
        py[p] = py[p - 1] * y;
        pz[p] = pz[p - 1] * z;
    }
#pragma unroll
    for (int q = 0; q < NLM; q++) S[q] = 0.0;
#pragma unroll
    for (int t = 0; t < N_MONO_TERMS; t++) {
        const Mono m = c_mono[t];
        S[m.lm] = fma(m.coef, px[m.a] * py[m.b] * pz[m.c], S[m.lm]);
    }
}

// ---------------------------------------------------------------- sphere records
// rec[i][*]: 0-2 pos, 3 R, 4-6 W_k, 7-9 zeta_k, 10-12 A_k, 13-15 B_k, 16-18 (a, b, c),
// 19 q, 20 rho0(R), 21 rho0'(R), 22-23: x y z R^2 as four floats, 24-47: c_lm / R^l as 24
// double-floats (float pairs)
enum { RX = 0, RR = 3, RW = 4, RZ = 7, RA = 10, RB = 13, RC = 16, RQ = 19, RRHO = 20, RDRHO = 21, RXF = 22, RNS = 24 };

struct SphArgs {
    int na;
    const double *pos, *Z, *R, *w, *zeta, *clm;
    const double* ax[3];
    int n[3];
    double* rec;
    double *q, *rhoR, *drhoR, *coef;
    int* status;
};

constexpr int SPH_NT = 128;

__global__ void __launch_bounds__(SPH_NT) k_sphere_params(SphArgs a)
{
    __shared__ double sm[32];
    __shared__ double red[6];
    __shared__ int bad_geom, bad_zeta;
    const int i = blockIdx.x;
    if (threadIdx.x == 0) bad_geom = bad_zeta = 0;
    __syncthreads();
    const double xi = a.pos[3 * i], yi = a.pos[3 * i + 1], zi = a.pos[3 * i + 2], Ri = a.R[i];
    double zt[3];
    for (int k = 0; k < 3; k++) zt[k] = a.zeta[3 * i + k];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < a.na; j += SPH_NT) {
        if (j == i) continue;
        const double dx = a.pos[3 * j] - xi, dy = a.pos[3 * j + 1] - yi, dz = a.pos[3 * j + 2] - zi;
        const double D = sqrt(dx * dx + dy * dy + dz * dz);
        if (!(D >= Ri + a.R[j])) bad_geom = 1;
        for (int k = 0; k < 3; k++) {
            const double z = a.zeta[3 * j + k];
            if (z != zt[k]) bad_zeta = 1;
            const double W = a.w[3 * j + k] * z * z * z / (8.0 * PI);
            const double e = exp(-z * D);
            acc[k] += W * e * (1.0 + z * D) / (2.0 * D * z * z);
            acc[3 + k] += W * e / (2.0 * D * z);
        }
    }
    for (int v = 0; v < 6; v++) {
        const double s = block_sum<SPH_NT>(acc[v], sm);
        if (threadIdx.x == 0) red[v] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    // the sphere must sit two nodes inside every face
    for (int d = 0; d < 3; d++) {
        const double c = a.pos[3 * i + d];
        if (!(c - Ri >= a.ax[d][2] && c + Ri <= a.ax[d][a.n[d] - 3])) bad_geom = 1;
    }
    double* r = a.rec + (size_t)SPHERE_REC_DOUBLES * i;
    r[RX] = xi;
    r[RX + 1] = yi;
    r[RX + 2] = zi;
    r[RR] = Ri;
    {
        float* xf = reinterpret_cast<float*>(r + RXF);
        xf[0] = (float)xi;
        xf[1] = (float)yi;
        xf[2] = (float)zi;
        xf[3] = (float)(Ri * Ri);
    }
    double rho = 0.0, drho = 0.0, inside = 0.0;
    for (int k = 0; k < 3; k++) {
        const double z = zt[k], wk = a.w[3 * i + k];
        const double W = wk * z * z * z / (8.0 * PI);
        const double A = red[k], B = red[3 + k];
        r[RW + k] = W;
        r[RZ + k] = z;
        r[RA + k] = A;
        r[RB + k] = B;
        const double zR = z * Ri, eR = exp(-zR), sh = sinh(zR), ch = cosh(zR);
        rho += W * eR + 2.0 * A * sh / Ri - 2.0 * B * ch;
        drho += -z * W * eR + 2.0 * A * (z * ch / Ri - sh / (Ri * Ri)) - 2.0 * B * z * sh;
        // electrons inside the sphere: own normalised Slater term + neighbour averages
        const double own = wk * (1.0 - eR * (1.0 + zR + 0.5 * zR * zR));
        const double I1 = Ri * ch / z - sh / (z * z);                                   // int r sinh
        const double I2 = Ri * Ri * sh / z - 2.0 * Ri * ch / (z * z) + 2.0 * sh / (z * z * z);  // int r^2 cosh
        inside += own + 4.0 * PI * (2.0 * A * I1 - 2.0 * B * I2);
    }
    const double q = inside - a.Z[i];
    const double Qr = q / (4.0 * PI);
    const double R2 = Ri * Ri, R3 = R2 * Ri, R4 = R2 * R2, R7 = R4 * R3;
    const double cc = (Qr - rho * R3 / 3.0 + drho * R4 / 15.0) * (105.0 / (8.0 * R7));
    const double bb = drho / (2.0 * Ri) - 2.0 * cc * R2;
    const double aa = rho - 0.5 * drho * Ri + cc * R4;
    r[RC] = aa;
    r[RC + 1] = bb;
    r[RC + 2] = cc;
    r[RQ] = q;
    r[RRHO] = rho;
    r[RDRHO] = drho;
    {
        float* ns = reinterpret_cast<float*>(r + RNS);
        double iRl = 1.0;
        int l = 0;
        for (int lm = 1; lm < NLM; lm++) {
            const int ll = l_of_lm(lm);
            while (l < ll) {
                iRl /= Ri;
                l++;
            }
            const double v = a.clm[24 * (size_t)i + lm - 1] * iRl;
            ns[2 * (lm - 1)] = (float)v;
            ns[2 * (lm - 1) + 1] = (float)(v - (double)(float)v);
        }
    }
    if (a.q) a.q[i] = q;
    if (a.rhoR) a.rhoR[i] = rho;
    if (a.drhoR) a.drhoR[i] = drho;
    if (a.coef) {
        a.coef[3 * i] = aa;
        a.coef[3 * i + 1] = bb;
        a.coef[3 * i + 2] = cc;
    }
    if (a.status) {
        if (bad_zeta) atomicMax(a.status, (int)LASTO_ERR_INVALID_ARG);
        if (bad_geom) atomicMax(a.status, (int)LASTO_ERR_GEOMETRY);
    }
}

cudaError_t launch_sphere_params(const lasto_cluster& cl, const double* ax0, const double* ax1, const double* ax2,
                                 double* rec, double* q, double* rhoR, double* drhoR, double* coef, int* status,
                                 cudaStream_t s)
{
    SphArgs a;
    a.na = cl.n_atoms;
    a.pos = cl.pos;
    a.Z = cl.Z;
    a.R = cl.R;
    a.w = cl.slater_w;
    a.zeta = cl.slater_zeta;
    a.clm = cl.c_lm;
    a.ax[0] = ax0;
    a.ax[1] = ax1;
    a.ax[2] = ax2;
    for (int d = 0; d < 3; d++) a.n[d] = cl.n[d];
    a.rec = rec;
    a.q = q;
    a.rhoR = rhoR;
    a.drhoR = drhoR;
    a.coef = coef;
    a.status = status;
    k_sphere_params<<<cl.n_atoms, SPH_NT, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- deposit (FP64)
struct DepArgs {
    int na;
    int n[3];
    const double* ax[3];
    const double* rec;
    const double* clm;
    double* b;
    int* owner;
    int* status;
};

// FP32-pair deposit, per atom floats: {D(x,y,z) rounded to FP32, R^2}, {W_k rounded to FP32, 0},
// then the double-float D(x,y,z) and W_k pairs (D = atom - tile origin)
constexpr int SAF = 20;
__global__ void k_deposit_df(DepArgs a);

// per-atom fields staged in shared memory
constexpr int SA = 14;  // x y z R^2 W0 W1 W2 A0 A1 A2 B0 B1 B2 R
constexpr int DEP_NT = 256;
constexpr int DT_X = 8, DT_Y = 8, DT_Z = 4;   // FP32-pair deposit: one 8 x 8 x 4 tile of nodes per block
static_assert(DT_X * DT_Y * DT_Z == DEP_NT, "deposit tile = one block");
constexpr double EXP_CUT = 40.0;   // e^{-40} * max W < 1e-14 absolute; skipped terms are below FP64 rounding of n_e
// FP32-pair deposit: Slater terms with zeta r > FAR_T in plain FP32.  FP32 carries a relative
// error of a few 1e-6 in e^{-zeta r} there (the FP32 distance and exponent); at 20 the node-wise
// deposit error stays near 1e-10 of the local density, while 16 (measured) raises it to ~4e-9.
constexpr float FAR_T = 20.0f;
// FP32-pair deposit: Slater terms with zeta r > DF_EXP_CUT are dropped, and atoms beyond
// DF_EXP_CUT / zeta_min of a tile's bounding box for the whole tile.  Measured against the
// oracle on the small test clusters (Pd13 graded 33^3 and uniform 65^3, Pd2): the largest
// node-wise error where the density exceeds 1e-3 of its maximum is 2e-11 to 6e-11 of the local
// density at 37 (FP32 far field included); at 34 it was 3.6e-10.
constexpr float DF_EXP_CUT = 37.0f;

__device__ __forceinline__ double nonspherical(const double* __restrict__ c, double dx, double dy, double dz,
                                               double r, double R, double z1)
{
    double S[NLM];
    solid_harmonics(dx, dy, dz, S);
    const double iR = 1.0 / R;
    double ang = 0.0, Rl = iR;
    int l = 1;
    for (int lm = 1; lm < NLM; lm++) {
        const int ll = l_of_lm(lm);
        if (ll != l) {
            Rl *= iR;
            l = ll;
        }
        ang = fma(c[lm - 1] * Rl, S[lm], ang);
    }
    const double t = 1.0 - r * r * iR * iR;
    return z1 * z1 * z1 / (8.0 * PI) * exp(-z1 * r) * t * t * ang;
}

__global__ void __launch_bounds__(DEP_NT) k_deposit64(DepArgs a)
{
    extern __shared__ double sat[];
    // the exponents are the same on every atom (checked by the sphere kernel): take atom 0's
    const double z0 = a.rec[RZ], z1 = a.rec[RZ + 1], z2 = a.rec[RZ + 2];
    for (int t = threadIdx.x; t < a.na; t += DEP_NT) {
        const double* r = a.rec + (size_t)SPHERE_REC_DOUBLES * t;
        double* o = sat + SA * t;
        o[0] = r[RX];
        o[1] = r[RX + 1];
        o[2] = r[RX + 2];
        o[3] = r[RR] * r[RR];
        for (int k = 0; k < 3; k++) {
            o[4 + k] = r[RW + k];
            o[7 + k] = r[RA + k];
            o[10 + k] = r[RB + k];
        }
        o[13] = r[RR];
    }
    __syncthreads();
    const size_t N = (size_t)a.n[0] * a.n[1] * a.n[2];
    const size_t P = blockIdx.x * (size_t)DEP_NT + threadIdx.x;
    if (P >= N) return;
    const size_t nxy = (size_t)a.n[0] * a.n[1];
    const int k = (int)(P / nxy);
    const int j = (int)((P - (size_t)k * nxy) / a.n[0]);
    const int i = (int)(P - (size_t)k * nxy - (size_t)j * a.n[0]);
    const double x = a.ax[0][i], y = a.ax[1][j], z = a.ax[2][k];
    const double zz[3] = {z0, z1, z2};
    double s = 0.0;
    int own = -1;
    double ox = 0, oy = 0, oz = 0, or2 = 0;
    for (int t = 0; t < a.na; t++) {
        const double* o = sat + SA * t;
        const double dx = x - o[0], dy = y - o[1], dz = z - o[2];
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        if (r2 < o[3]) {
            own = t;
            ox = dx;
            oy = dy;
            oz = dz;
            or2 = r2;
            continue;
        }
        const double r = sqrt(r2);
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const double e = zz[q] * r;
            if (e < EXP_CUT) s = fma(o[4 + q], exp(-e), s);
        }
    }
    if (own >= 0) {
        const double* o = sat + SA * own;
        const double* rc = a.rec + (size_t)SPHERE_REC_DOUBLES * own;
        const double r = sqrt(or2);
        double nbr = 0.0;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const double zr = zz[q] * r;
            const double shr = (zr > 1e-6) ? sinh(zr) / r : zz[q] * (1.0 + zr * zr / 6.0);
            nbr += 2.0 * o[7 + q] * shr - 2.0 * o[10 + q] * cosh(zr);
        }
        const double pseudo = fma(fma(rc[RC + 2], or2, rc[RC + 1]), or2, rc[RC]);
        const double ns = nonspherical(a.clm + 24 * (size_t)own, ox, oy, oz, r, o[13], z0);
        s = s - nbr + ns + pseudo;
    }
    const double bv = 4.0 * PI * s;
    a.b[P] = bv;
    if (a.owner) a.owner[P] = own;
    if (!isfinite(bv) && a.status) atomicMax(a.status, (int)LASTO_ERR_NONFINITE);
}


cudaError_t launch_deposit(const lasto_cluster& cl, const double* rec, int precision, double* b, int* owner,
                           const double* /*xm_tab*/, double* /*row_mom*/, int* status, cudaStream_t s)
{
    cudaError_t e = ensure_monomials();
    if (e != cudaSuccess) return e;
    DepArgs a;
    a.na = cl.n_atoms;
    for (int d = 0; d < 3; d++) a.n[d] = cl.n[d];
    a.ax[0] = cl.x;
    a.ax[1] = cl.y;
    a.ax[2] = cl.z;
    a.rec = rec;
    a.clm = cl.c_lm;
    a.b = b;
    a.owner = owner;
    a.status = status;
    const size_t N = (size_t)cl.n[0] * cl.n[1] * cl.n[2];
    const size_t smem = sizeof(double) * SA * (size_t)cl.n_atoms;
    if (precision == LASTO_PREC_MIXED) {
        const size_t smf = sizeof(float) * (128 + SAF * (size_t)cl.n_atoms) + sizeof(int) * (size_t)cl.n_atoms;
        if (smf > 200 * 1024) return cudaErrorInvalidValue;
        const dim3 grid((unsigned)((cl.n[0] + DT_X - 1) / DT_X), (unsigned)((cl.n[1] + DT_Y - 1) / DT_Y),
                        (unsigned)((cl.n[2] + DT_Z - 1) / DT_Z));
        if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
        k_deposit_df<<<grid, DEP_NT, smf, s>>>(a);
        return cudaGetLastError();
    }
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    k_deposit64<<<(unsigned)((N + DEP_NT - 1) / DEP_NT), DEP_NT, smem, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- deposit (FP32 pairs)
using dfa::df;

__device__ __forceinline__ bool inside_fp64(const DepArgs& a, double x, double y, double z, int t)
{
    const double* r = a.rec + (size_t)SPHERE_REC_DOUBLES * t;
    const double dx = x - r[RX], dy = y - r[RX + 1], dz = z - r[RX + 2];
    return fma(dx, dx, fma(dy, dy, dz * dz)) < r[RR] * r[RR];
}

// The FP32-pair deposit works on 8 x 8 x 4 tiles of nodes (a warp covers 8 x 4 x 1): a compact
// footprint lets a whole warp agree more often on which branch an atom takes (double-float,
// plain FP32 far field, beyond the cut-off), and lets the block drop, once, every atom whose
// distance from the tile's bounding box exceeds the cut-off (each node would skip it anyway).

__global__ void __launch_bounds__(DEP_NT) k_deposit_df(DepArgs a)
{
    extern __shared__ float sf[];
    __shared__ int s_cnt[DEP_NT / 32];
    __shared__ float s_off[2 * (DT_X + DT_Y + DT_Z)];   // node coordinate - tile origin, double-float
    float* th = sf;
    float* tl = sf + 64;
    float* sat = sf + 128;
    int* list = reinterpret_cast<int*>(sat + SAF * (size_t)a.na);
    const int i0 = blockIdx.x * DT_X, j0 = blockIdx.y * DT_Y, k0 = blockIdx.z * DT_Z;
    const int i = i0 + (threadIdx.x & 7), j = j0 + ((threadIdx.x >> 3) & 7), k = k0 + (threadIdx.x >> 6);
    const bool valid = i < a.n[0] && j < a.n[1] && k < a.n[2];
    // tile origin: its first node; offsets from it keep the pairs' magnitudes small
    const double ox = a.ax[0][i0], oy = a.ax[1][j0], oz = a.ax[2][k0];
    for (int t = threadIdx.x; t < 64; t += DEP_NT) {
        th[t] = c_exp_h[t];
        tl[t] = c_exp_l[t];
    }
    if (threadIdx.x < DT_X + DT_Y + DT_Z) {
        const int t = threadIdx.x;
        const int d = t < DT_X ? 0 : t < DT_X + DT_Y ? 1 : 2;
        const int o = t - (d == 0 ? 0 : d == 1 ? DT_X : DT_X + DT_Y);
        const int first = d == 0 ? i0 : d == 1 ? j0 : k0;
        const double org = d == 0 ? ox : d == 1 ? oy : oz;
        const df v = dfa::from_double(a.ax[d][min(first + o, a.n[d] - 1)] - org);
        s_off[2 * t] = v.h;
        s_off[2 * t + 1] = v.l;
    }
    df zt[3];
    float zmin = 1e30f;
    for (int q = 0; q < 3; q++) {
        zt[q] = dfa::from_double(a.rec[RZ + q]);
        zmin = fminf(zmin, zt[q].h);
    }
    const float cut = DF_EXP_CUT / zmin;
    const float cut2 = cut * cut * (1.0f + 1e-5f);
    int nkept, nnear;
    // Atoms within the cut-off of the tile's bounding box, in ascending order, tested in FP32
    // on the records' float copies of the positions: first those that may come within
    // FAR_T / zeta_min of a node of the tile (near candidates), then those farther than that
    // from every node (far-only).  The margins 1e-3 on the squared distances cover the
    // rounding of these tests (~1e-6 relative) and of a node's own FP32 distance tests, so an
    // atom dropped here fails the cut-off test, and a far-only atom passes the far test, at
    // every node of the tile.
    const float far_box2 = (FAR_T / zmin) * (FAR_T / zmin) * (1.0f + 1e-3f);
    {
        const float bx0 = (float)ox, bx1 = (float)a.ax[0][min(i0 + DT_X - 1, a.n[0] - 1)];
        const float by0 = (float)oy, by1 = (float)a.ax[1][min(j0 + DT_Y - 1, a.n[1] - 1)];
        const float bz0 = (float)oz, bz1 = (float)a.ax[2][min(k0 + DT_Z - 1, a.n[2] - 1)];
        const float lim = cut2 * (1.0f + 1e-3f);
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        int total = 0;
        for (int pass = 0; pass < 2; pass++) {
            if (pass == 1) nnear = total;
            for (int base = 0; base < a.na; base += DEP_NT) {
                const int t = base + threadIdx.x;
                bool keep = false;
                if (t < a.na) {
                    const float4 c = *reinterpret_cast<const float4*>(a.rec + (size_t)SPHERE_REC_DOUBLES * t + RXF);
                    const float ex = fmaxf(fmaxf(bx0 - c.x, c.x - bx1), 0.0f);
                    const float ey = fmaxf(fmaxf(by0 - c.y, c.y - by1), 0.0f);
                    const float ez = fmaxf(fmaxf(bz0 - c.z, c.z - bz1), 0.0f);
                    const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                    keep = d2 <= lim && ((d2 > far_box2) == (pass == 1));
                }
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if (l == 0) s_cnt[w] = __popc(m);
                __syncthreads();
                int off = total, sum = 0;
                for (int q = 0; q < DEP_NT / 32; q++) {
                    off += q < w ? s_cnt[q] : 0;
                    sum += s_cnt[q];
                }
                if (keep) list[off + __popc(m & ((1u << l) - 1u))] = t;
                __syncthreads();
                total += sum;
            }
        }
        // stage the kept atoms' fields in list order (far-only atoms: offsets and weights only,
        // {D(x,y,z), W_0} and {W_1, W_2}, the layout of their loop below)
        for (int q = threadIdx.x; q < total; q += DEP_NT) {
            const double* r = a.rec + (size_t)SPHERE_REC_DOUBLES * list[q];
            float* o = sat + SAF * q;
            if (q >= nnear) {
                o[0] = (float)(r[RX] - ox);
                o[1] = (float)(r[RX + 1] - oy);
                o[2] = (float)(r[RX + 2] - oz);
                o[3] = (float)r[RW];
                o[4] = (float)r[RW + 1];
                o[5] = (float)r[RW + 2];
                continue;
            }
            const df Dx = dfa::from_double(r[RX] - ox), Dy = dfa::from_double(r[RX + 1] - oy),
                     Dz = dfa::from_double(r[RX + 2] - oz);
            o[0] = Dx.h; o[1] = Dy.h; o[2] = Dz.h;
            o[3] = reinterpret_cast<const float*>(r + RXF)[3];
            o[8] = Dx.h; o[9] = Dx.l; o[10] = Dy.h; o[11] = Dy.l; o[12] = Dz.h; o[13] = Dz.l;
            for (int c = 0; c < 3; c++) {
                const df W = dfa::from_double(r[RW + c]);
                o[4 + c] = W.h;
                o[14 + 2 * c] = W.h;
                o[15 + 2 * c] = W.l;
            }
            o[7] = 0.0f;
        }
        __syncthreads();
        nkept = total;
    }
    if (!valid) return;
    const size_t P = ((size_t)k * a.n[1] + j) * a.n[0] + i;
    const double x = a.ax[0][i], y = a.ax[1][j], z = a.ax[2][k];
    const int li = threadIdx.x & 7, lj = DT_X + ((threadIdx.x >> 3) & 7), lk = DT_X + DT_Y + (threadIdx.x >> 6);
    const df px = {s_off[2 * li], s_off[2 * li + 1]}, py = {s_off[2 * lj], s_off[2 * lj + 1]},
             pz = {s_off[2 * lk], s_off[2 * lk + 1]};
    bool twice[3];   // zeta_q exactly twice zeta_0 (both parts of the double-float)
#pragma unroll
    for (int q = 0; q < 3; q++) twice[q] = q > 0 && zt[q].h == 2.0f * zt[0].h && zt[q].l == 2.0f * zt[0].l;
    // beyond zeta_min r = FAR_T every Slater term is below e^-20 of its weight: plain FP32
    // (relative error ~1e-7 of terms that small is ~1e-16 of the node's density scale)
    const float far = FAR_T / zmin;
    const float far2 = far * far * (1.0f + 1e-4f);
    df s = {0.0f, 0.0f};
    // the Slater terms beyond zeta r = FAR_T (each below e^-20 of its weight) summed in plain
    // FP32 and added to the double-float sum once: their total is below 1e-6 of the node's
    // density wherever that density matters, so FP32 rounding of it stays below 1e-13
    float sfar = 0.0f;
    int own = -1;
    df orr2 = {0.0f, 0.0f}, odx = s, ody = s, odz = s;
    for (int q0 = 0; q0 < nnear; q0++) {
        const float* o = sat + SAF * q0;
        // the pair's distance in FP32 from the FP32 roundings of the two offsets (one subtraction
        // per axis): the atom's offset is at most r + the tile's extent, so r carries a relative
        // error of ~1.5e-7 wherever the far field applies (r >= FAR_T / zeta_max)
        const float4 A = *reinterpret_cast<const float4*>(o);
        const float fx = px.h - A.x, fy = py.h - A.y, fz = pz.h - A.z;
        const float r2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
        if (r2f > cut2) continue;
        if (r2f > far2) {
            // far pair: every term is below e^-FAR_T of its weight; the ~1.5e-7 relative error of
            // r is ~3e-6 in e^{-zeta r} at zeta r = 20, the fast reciprocal square root and
            // exponential add errors of the same size, and e^{-zeta_q r} for zeta_q = 2 zeta_0
            // is the square of e^{-zeta_0 r}.  Terms beyond zeta r = DF_EXP_CUT are dropped.
            const float4 W = *reinterpret_cast<const float4*>(o + 4);
            const float rf = r2f * rsqrtf(r2f);
            const float e0 = __expf(-zt[0].h * rf);
            sfar = fmaf(W.x, e0, sfar);
            if (twice[1]) {
                sfar = fmaf(W.y, e0 * e0, sfar);
            } else {
                const float e = zt[1].h * rf;
                if (e < DF_EXP_CUT) sfar = fmaf(W.y, __expf(-e), sfar);
            }
            if (twice[2]) {
                sfar = fmaf(W.z, e0 * e0, sfar);
            } else {
                const float e = zt[2].h * rf;
                if (e < DF_EXP_CUT) sfar = fmaf(W.z, __expf(-e), sfar);
            }
            continue;
        }
        const df dx = dfa::add(px, df{-o[8], -o[9]});
        const df dy = dfa::add(py, df{-o[10], -o[11]});
        const df dz = dfa::add(pz, df{-o[12], -o[13]});
        const df r2 = dfa::add(dfa::add(dfa::sqr(dx), dfa::sqr(dy)), dfa::sqr(dz));
        if (r2.h > cut2) continue;
        if (r2.h < A.w * (1.0f + 2e-6f)) {
            const int t = list[q0];
            const bool in = (r2.h < A.w * (1.0f - 2e-6f)) ? true : inside_fp64(a, x, y, z, t);
            if (in) {
                own = t;
                orr2 = r2;
                odx = dx;
                ody = dy;
                odz = dz;
                continue;
            }
        }
        const df r = dfa::sqrt_df(r2);
        df e0 = {0.0f, 0.0f};   // e^{-zeta_0 r} when it was taken in double-float
        bool have0 = false;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const df tq = dfa::mul(r, zt[q]);
            if (tq.h >= DF_EXP_CUT) continue;
            if (tq.h > FAR_T) {
                sfar = fmaf(o[14 + 2 * q], expf(-tq.h), sfar);
            } else {
                // zeta_q = 2 zeta_0 (as in the density model's 1.5, 3.0): e^{-zeta_q r} = (e^{-zeta_0 r})^2
                const df eq = (q > 0 && twice[q] && have0) ? dfa::sqr(e0) : dfa::exp_neg(tq, th, tl);
                if (q == 0) {
                    e0 = eq;
                    have0 = true;
                }
                s = dfa::add(s, dfa::mul(df{o[14 + 2 * q], o[15 + 2 * q]}, eq));
            }
        }
    }
    // far-only atoms: every node of the tile is beyond FAR_T / zeta_min of them, so only the
    // far-field terms remain, and a term whose exponent exceeds DF_EXP_CUT at that distance
    // (zeta_q >= zeta_min DF_EXP_CUT / FAR_T) is dropped for all of them at once
    {
        bool qf[3];
#pragma unroll
        for (int q = 0; q < 3; q++) qf[q] = zt[q].h * (FAR_T / zmin) < DF_EXP_CUT;
        const float z0 = zt[0].h, z1 = zt[1].h, z2 = zt[2].h;
        for (int q0 = nnear; q0 < nkept; q0++) {
            const float* o = sat + SAF * q0;
            const float4 A = *reinterpret_cast<const float4*>(o);
            const float fx = px.h - A.x, fy = py.h - A.y, fz = pz.h - A.z;
            const float r2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
            const float rf = r2f * rsqrtf(r2f);
            if (qf[0]) sfar = fmaf(A.w, __expf(-z0 * rf), sfar);
            if (qf[1]) sfar = fmaf(o[4], __expf(-z1 * rf), sfar);
            if (qf[2]) sfar = fmaf(o[5], __expf(-z2 * rf), sfar);
        }
    }
    if (own >= 0) {
        const double* rc = a.rec + (size_t)SPHERE_REC_DOUBLES * own;
        const df r = dfa::sqrt_df(orr2);
        df nbr = {0.0f, 0.0f}, e1 = {1.0f, 0.0f};
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const df zr = dfa::mul(r, zt[q]);
            const df em = dfa::exp_neg(zr, th, tl), ep = dfa::exp_neg(dfa::neg(zr), th, tl);
            if (q == 0) e1 = em;
            df shr;   // sinh(zeta r) / r
            if (zr.h > 1e-3f) {
                df sh = dfa::add(ep, dfa::neg(em));
                sh.h *= 0.5f;
                sh.l *= 0.5f;
                shr = dfa::div(sh, r);
            } else {
                shr = dfa::mul(zt[q], dfa::add_f(df{1.0f, 0.0f}, zr.h * zr.h * (1.0f / 6.0f)));
            }
            df ch = dfa::add(ep, em);
            ch.h *= 0.5f;
            ch.l *= 0.5f;
            const df A2 = dfa::from_double(2.0 * rc[RA + q]), B2 = dfa::from_double(2.0 * rc[RB + q]);
            nbr = dfa::add(nbr, dfa::add(dfa::mul(A2, shr), dfa::neg(dfa::mul(B2, ch))));
        }
        const df ca = dfa::from_double(rc[RC]), cb = dfa::from_double(rc[RC + 1]), cc = dfa::from_double(rc[RC + 2]);
        const df pseudo = dfa::add(ca, dfa::mul(orr2, dfa::add(cb, dfa::mul(orr2, cc))));
        // nonspherical part: slater(zeta_1, r) (1 - r^2/R^2)^2 sum c_lm (r/R)^l y_lm
        const float* ns = reinterpret_cast<const float*>(rc + RNS);
        df pxs[5], pys[5], pzs[5];
        pxs[0] = pys[0] = pzs[0] = df{1.0f, 0.0f};
        for (int p = 1; p < 5; p++) {
            pxs[p] = dfa::mul(pxs[p - 1], odx);
            pys[p] = dfa::mul(pys[p - 1], ody);
            pzs[p] = dfa::mul(pzs[p - 1], odz);
        }
        df ang = {0.0f, 0.0f};
        for (int t = 1; t < N_MONO_TERMS; t++) {
            const MonoF m = c_mono_f[t];
            const df term = dfa::mul(dfa::mul(df{m.h, m.l}, df{ns[2 * (m.lm - 1)], ns[2 * (m.lm - 1) + 1]}),
                                     dfa::mul(dfa::mul(pxs[m.a], pys[m.b]), pzs[m.c]));
            ang = dfa::add(ang, term);
        }
        const double R = rc[RR];
        const df invR2 = dfa::from_double(1.0 / (R * R));
        const df tt = dfa::add_f(dfa::neg(dfa::mul(orr2, invR2)), 1.0f);
        const double z1 = rc[RZ];
        const df radial = dfa::mul(dfa::mul(dfa::from_double(z1 * z1 * z1 / (8.0 * PI)), e1), dfa::sqr(tt));
        const df nsv = dfa::mul(radial, ang);
        s = dfa::add(dfa::add(s, dfa::neg(nbr)), dfa::add(pseudo, nsv));
    }
    s = dfa::add_f(s, sfar);
    const df fourpi = dfa::from_double(4.0 * PI);
    const double bv = dfa::to_double(dfa::mul(fourpi, s));
    a.b[P] = bv;
    if (a.owner) a.owner[P] = own;
    if (!isfinite(bv) && a.status) atomicMax(a.status, (int)LASTO_ERR_NONFINITE);
}

void init_device_constants()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return;
    {
        std::lock_guard<std::mutex> lock(g_constants_mutex);
        if (g_constants_done[dev]) return;
    }
    ensure_monomials();
    cudaFuncSetAttribute(k_deposit64, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_deposit_df, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    init_mg_attributes();
    init_slab_attributes();
    init_wave_attributes();
    std::lock_guard<std::mutex> lock(g_constants_mutex);
    g_constants_done[dev] = true;
}

// ---------------------------------------------------------------- boundary multipoles
// Q_lm = sum (b/4pi) vol S_lm(node - centre).  S_lm is a polynomial of degree l in
// (x, y, z) and vol a product of per-axis dual lengths, so the sum factorises:
// per-row x-moments (5 FMAs per node), then y and z contractions over the rows,
// then the monomial expansion of each S_lm.
constexpr int MOM_NT = 128;

// xm[a][i] = (x_i - cx)^a * dual_i, a = 0..4
__global__ void k_moment_table(const double* __restrict__ x, int n, double c, double* __restrict__ tab)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dual = (i == 0) ? 0.5 * (x[1] - x[0]) : (i == n - 1) ? 0.5 * (x[n - 1] - x[n - 2])
                                                                  : 0.5 * (x[i + 1] - x[i - 1]);
    const double d = x[i] - c;
    double p = dual;
    for (int a = 0; a < 5; a++) {
        tab[(size_t)a * n + i] = p;
        p *= d;
    }
}

// row_mom[a][row] = sum_i xm[a][i] b[row, i],  row = k*ny + j: one thread per row, sequential
// FP64 sums (no shuffle trees: FP64 adds are scarce on this GPU).
__global__ void __launch_bounds__(MOM_NT) k_row_moments(const double* __restrict__ b, int nx, size_t nrows,
                                                       const double* __restrict__ xm, double* __restrict__ row_mom)
{
    const size_t row = blockIdx.x * (size_t)MOM_NT + threadIdx.x;
    if (row >= nrows) return;
    const double* br = b + row * nx;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int i = 0; i < nx; i++) {
        const double v = br[i];
#pragma unroll
        for (int q = 0; q < 5; q++) acc[q] = fma(xm[(size_t)q * nx + i], v, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 5; q++) row_mom[(size_t)q * nrows + row] = acc[q];
}

// pairs (a, b) with a + b <= 4, in a fixed order
__constant__ int c_ab[15][2] = {{0, 0}, {0, 1}, {0, 2}, {0, 3}, {0, 4}, {1, 0}, {1, 1}, {1, 2}, {1, 3},
                                {2, 0}, {2, 1}, {2, 2}, {3, 0}, {3, 1}, {4, 0}};

// plane[ab][k] = sum_j ym[b][j] row_mom[a][k*ny + j]: one thread per (ab, k)
__global__ void __launch_bounds__(MOM_NT) k_plane_moments(const double* __restrict__ row_mom, int ny, int nz,
                                                         const double* __restrict__ ym, double* __restrict__ plane)
{
    const int t = blockIdx.x * MOM_NT + threadIdx.x;
    if (t >= 15 * nz) return;
    const int ab = t / nz, k = t - ab * nz;
    const int A = c_ab[ab][0], B = c_ab[ab][1];
    const size_t nrows = (size_t)ny * nz;
    const double* rm = row_mom + (size_t)A * nrows + (size_t)k * ny;
    const double* yb = ym + (size_t)B * ny;
    double acc = 0.0;
    for (int j = 0; j < ny; j++) acc = fma(yb[j], rm[j], acc);
    plane[(size_t)ab * nz + k] = acc;
}

// M[a][b][c] = sum_k zm[c][k] plane[ab][k] (one thread per monomial); Q_lm = sum_terms coef M / (4 pi)
__global__ void __launch_bounds__(64) k_final_moments(const double* __restrict__ plane, int nz,
                                                     const double* __restrict__ zm, double* __restrict__ Q)
{
    __shared__ double M[5][5][5];
    const int t = threadIdx.x;
    if (t < 35) {
        // monomial t -> (ab, c) in the order of c_ab with c = 0 .. 4 - a - b
        int idx = 0, ab = 0, C = 0;
        for (int q = 0; q < 15; q++) {
            const int room = 5 - c_ab[q][0] - c_ab[q][1];
            if (t < idx + room) {
                ab = q;
                C = t - idx;
                break;
            }
            idx += room;
        }
        double acc = 0.0;
        const double* pl = plane + (size_t)ab * nz;
        const double* zc = zm + (size_t)C * nz;
        for (int k = 0; k < nz; k++) acc = fma(zc[k], pl[k], acc);
        M[c_ab[ab][0]][c_ab[ab][1]][C] = acc;
    }
    __syncthreads();
    if (t < NLM) {
        double q = 0.0;
        for (int m = 0; m < N_MONO_TERMS; m++) {
            const Mono mo = c_mono[m];
            if (mo.lm == t) q = fma(mo.coef, M[mo.a][mo.b][mo.c], q);
        }
        Q[t] = q / (4.0 * PI);
    }
}

cudaError_t launch_multipoles(const int n[3], const double* x, const double* y, const double* z, const double* b,
                              const double centre[3], double* tabs, double* row_mom, double* plane, double* Q,
                              cudaStream_t s)
{
    cudaError_t e = ensure_monomials();
    if (e != cudaSuccess) return e;
    double* xm = tabs;
    double* ym = xm + 5 * (size_t)n[0];
    double* zm = ym + 5 * (size_t)n[1];
    k_moment_table<<<(n[0] + 127) / 128, 128, 0, s>>>(x, n[0], centre[0], xm);
    k_moment_table<<<(n[1] + 127) / 128, 128, 0, s>>>(y, n[1], centre[1], ym);
    k_moment_table<<<(n[2] + 127) / 128, 128, 0, s>>>(z, n[2], centre[2], zm);
    const size_t nrows = (size_t)n[1] * n[2];
    k_row_moments<<<(unsigned)((nrows + MOM_NT - 1) / MOM_NT), MOM_NT, 0, s>>>(b, n[0], nrows, xm, row_mom);
    k_plane_moments<<<(15 * n[2] + MOM_NT - 1) / MOM_NT, MOM_NT, 0, s>>>(row_mom, n[1], n[2], ym, plane);
    k_final_moments<<<1, 64, 0, s>>>(plane, n[2], zm, Q);
    return cudaGetLastError();
}

size_t multipole_scratch_doubles(const int n[3])
{
    return 5 * ((size_t)n[0] + n[1] + n[2]) + 5 * (size_t)n[1] * n[2] + 15 * (size_t)n[2];
}

// ---------------------------------------------------------------- Dirichlet faces
// u = -sum_lm 4 pi/(2l+1) Q_lm S_lm(d) / r^(2l+1), d = node - centre (Eq. 2.7 decay).
__global__ void k_boundary_fill(int nx, int ny, int nz, const double* __restrict__ x, const double* __restrict__ y,
                                const double* __restrict__ z, double cx, double cy, double cz,
                                const double* __restrict__ Q, double* __restrict__ u)
{
    const size_t fx = (size_t)ny * nz, fy = (size_t)nx * nz, fz = (size_t)nx * ny;
    const size_t total = 2 * (fx + fy + fz);
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    size_t r = t;
    if (r < 2 * fx) {
        const int side = (int)(r / fx);
        r %= fx;
        i = side ? nx - 1 : 0;
        j = (int)(r % ny);
        k = (int)(r / ny);
    } else if ((r -= 2 * fx) < 2 * fy) {
        const int side = (int)(r / fy);
        r %= fy;
        j = side ? ny - 1 : 0;
        i = (int)(r % nx);
        k = (int)(r / nx);
    } else {
        r -= 2 * fy;
        const int side = (int)(r / fz);
        r %= fz;
        k = side ? nz - 1 : 0;
        i = (int)(r % nx);
        j = (int)(r / nx);
    }
    const double dx = x[i] - cx, dy = y[j] - cy, dz = z[k] - cz;
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double ir = 1.0 / sqrt(r2), ir2 = ir * ir;
    double S[NLM];
    solid_harmonics(dx, dy, dz, S);
    double v = 0.0, pw = ir;   // ir^(2l+1)
    int l = 0;
    for (int lm = 0; lm < NLM; lm++) {
        const int ll = l_of_lm(lm);
        if (ll != l) {
            pw *= ir2;
            l = ll;
        }
        v = fma(-4.0 * PI / (2.0 * l + 1.0) * Q[lm] * pw, S[lm], v);
    }
    u[((size_t)k * ny + j) * nx + i] = v;
}

cudaError_t launch_boundary_fill(const int n[3], const double* x, const double* y, const double* z, double cx,
                                 double cy, double cz, const double* Q, double* u, cudaStream_t s)
{
    cudaError_t e = ensure_monomials();
    if (e != cudaSuccess) return e;
    const size_t total = 2 * ((size_t)n[1] * n[2] + (size_t)n[0] * n[2] + (size_t)n[0] * n[1]);
    k_boundary_fill<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(n[0], n[1], n[2], x, y, z, cx, cy, cz, Q, u);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- exact superposition faces
// M_l = int_0^R zeta_1^3/(8pi) e^{-zeta_1 r} (1 - r^2/R^2)^2 (r/R)^l r^(l+2) dr, l = 0..4, by a
// 64-point Gauss-Legendre rule: block = atom, thread = node (found by Newton's method on the
// Legendre recurrence).
__global__ void k_nonsph_moments(int na, const double* __restrict__ R, const double* __restrict__ zeta,
                                 double* __restrict__ M)
{
    __shared__ double part[5][64];
    const int a = blockIdx.x, q = threadIdx.x;
    // node q of the 64-point rule (ascending cos), initial guess from the Chebyshev nodes
    double t = -cos(PI * (q + 0.75) / (64 + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; it++) {
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= 64; k++) {
            const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = 64 * (t * p1 - p0) / (t * t - 1.0);
        const double dt = p1 / dp;
        t -= dt;
        if (fabs(dt) < 1e-16) break;
    }
    const double wq = 2.0 / ((1.0 - t * t) * dp * dp);
    const double Ra = R[a], z1 = zeta[3 * a];
    const double r = 0.5 * Ra * (t + 1.0), tt = 1.0 - r * r / (Ra * Ra);
    const double f = 0.5 * Ra * wq * z1 * z1 * z1 / (8.0 * PI) * exp(-z1 * r) * tt * tt * r * r;
    double pl = 1.0;
    for (int l = 0; l < 5; l++) {
        part[l][q] = f * pl;
        pl *= (r / Ra) * r;
    }
    __syncthreads();
    for (int st = 32; st > 0; st >>= 1) {
        if (q < st)
            for (int l = 0; l < 5; l++) part[l][q] += part[l][q + st];
        __syncthreads();
    }
    if (q < 5) M[5 * (size_t)a + q] = part[q][0];
}

// u on the faces = sum over atoms of Z/r - sum_k w_k [1/r - e^{-zeta_k r}(1/r + zeta_k/2)]
// - sum_{l>=1,m} 4pi/(2l+1) c_lm M_l S_lm(d) / r^(2l+1), evaluated per atom as
// (Z - sum_k w_k)/r + sum_k w_k e^{-zeta_k r}(1/r + zeta_k/2) - sum_l r^-(2l+1) P_l(d), where
// P_l = sum_m 4pi/(2l+1) c_lm M_l S_lm is a homogeneous polynomial of degree l whose monomial
// coefficients each block forms once per atom (34 for l = 1..4).  Terms with zeta_k r >= 40
// (below e^-40 of w_k) are dropped, as in the deposit.
constexpr int EX_NT = 128;
constexpr int EX_CH = 64;        // atoms staged per pass
constexpr int EX_NC = 34;        // monomials of degree 1..4
constexpr int EX_REC = 10 + EX_NC;  // x y z q w0 w1 w2 zeta0 zeta1 zeta2 | coefficients

// slot of x^a y^b z^c (a + b + c = l, 1 <= l <= 4): degree offset + s(s+1)/2 + c, s = b + c
__host__ __device__ constexpr int ex_slot(int l, int b, int c)
{
    return (l == 1 ? 0 : l == 2 ? 3 : l == 3 ? 9 : 19) + (b + c) * (b + c + 1) / 2 + c;
}

__global__ void __launch_bounds__(EX_NT) k_boundary_exact(int nx, int ny, int nz, const double* __restrict__ x,
                                                          const double* __restrict__ y, const double* __restrict__ z,
                                                          int na, const double* __restrict__ pos,
                                                          const double* __restrict__ Zn, const double* __restrict__ w,
                                                          const double* __restrict__ zeta,
                                                          const double* __restrict__ clm,
                                                          const double* __restrict__ M, double* __restrict__ u)
{
    __shared__ double rec[EX_CH][EX_REC];
    const size_t fx = (size_t)ny * nz, fy = (size_t)nx * nz, fz = (size_t)nx * ny;
    const size_t total = 2 * (fx + fy + fz);
    const size_t t = blockIdx.x * (size_t)EX_NT + threadIdx.x;
    const bool valid = t < total;
    int i = 0, j = 0, k = 0;
    if (valid) {
        size_t r = t;
        if (r < 2 * fx) {
            const int side = (int)(r / fx);
            r %= fx;
            i = side ? nx - 1 : 0;
            j = (int)(r % ny);
            k = (int)(r / ny);
        } else if ((r -= 2 * fx) < 2 * fy) {
            const int side = (int)(r / fy);
            r %= fy;
            j = side ? ny - 1 : 0;
            i = (int)(r % nx);
            k = (int)(r / nx);
        } else {
            r -= 2 * fy;
            const int side = (int)(r / fz);
            r %= fz;
            k = side ? nz - 1 : 0;
            i = (int)(r % nx);
            j = (int)(r / nx);
        }
    }
    const double px = x[i], py = y[j], pz = z[k];
    double v = 0.0;
    for (int base = 0; base < na; base += EX_CH) {
        const int nch = min(EX_CH, na - base);
        __syncthreads();
        for (int q = threadIdx.x; q < nch; q += EX_NT) {
            const int at = base + q;
            double* o = rec[q];
            o[0] = pos[3 * at];
            o[1] = pos[3 * at + 1];
            o[2] = pos[3 * at + 2];
            o[3] = Zn[at] - (w[3 * at] + w[3 * at + 1] + w[3 * at + 2]);
            o[4] = w[3 * at];
            o[5] = w[3 * at + 1];
            o[6] = w[3 * at + 2];
            o[7] = zeta[3 * at];
            o[8] = zeta[3 * at + 1];
            o[9] = zeta[3 * at + 2];
            for (int c = 0; c < EX_NC; c++) o[10 + c] = 0.0;
            for (int tm = 1; tm < N_MONO_TERMS; tm++) {
                const Mono mo = c_mono[tm];
                const int l = l_of_lm(mo.lm);
                const double K = 4.0 * PI / (2 * l + 1) * clm[24 * (size_t)at + mo.lm - 1] * M[5 * (size_t)at + l];
                o[10 + ex_slot(l, mo.b, mo.c)] += K * mo.coef;
            }
        }
        __syncthreads();
        if (!valid) continue;
        for (int q = 0; q < nch; q++) {
            const double* o = rec[q];
            const double dx = px - o[0], dy = py - o[1], dz = pz - o[2];
            const double d = sqrt(fma(dx, dx, fma(dy, dy, dz * dz))), id = 1.0 / d, id2 = id * id;
            double e = o[3] * id;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const double zc = o[7 + c];
                if (zc * d < EXP_CUT) e = fma(o[4 + c] * exp(-zc * d), id + 0.5 * zc, e);
            }
            double xp[5], yp[5], zp[5];
            xp[0] = yp[0] = zp[0] = 1.0;
#pragma unroll
            for (int p = 1; p < 5; p++) {
                xp[p] = xp[p - 1] * dx;
                yp[p] = yp[p - 1] * dy;
                zp[p] = zp[p - 1] * dz;
            }
            double P[5];
#pragma unroll
            for (int l = 1; l <= 4; l++) {
                double acc = 0.0;
#pragma unroll
                for (int sb = 0; sb <= l; sb++)
#pragma unroll
                    for (int c = 0; c <= sb; c++)
                        acc = fma(o[10 + ex_slot(l, sb - c, c)], xp[l - sb] * yp[sb - c] * zp[c], acc);
                P[l] = acc;
            }
            const double multi = id2 * id * fma(id2, fma(id2, fma(id2, P[4], P[3]), P[2]), P[1]);
            v += e - multi;
        }
    }
    if (valid) u[((size_t)k * ny + j) * nx + i] = v;
}

cudaError_t launch_boundary_exact(const lasto_cluster& cl, double* M, double* u, cudaStream_t s)
{
    cudaError_t e = ensure_monomials();
    if (e != cudaSuccess) return e;
    k_nonsph_moments<<<cl.n_atoms, 64, 0, s>>>(cl.n_atoms, cl.R, cl.slater_zeta, M);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int* n = cl.n;
    const size_t total = 2 * ((size_t)n[1] * n[2] + (size_t)n[0] * n[2] + (size_t)n[0] * n[1]);
    k_boundary_exact<<<(unsigned)((total + EX_NT - 1) / EX_NT), EX_NT, 0, s>>>(n[0], n[1], n[2], cl.x, cl.y, cl.z, cl.n_atoms,
                                                                     cl.pos, cl.Z, cl.slater_w, cl.slater_zeta,
                                                                     cl.c_lm, M, u);
    return cudaGetLastError();
}

}  // namespace lasto
