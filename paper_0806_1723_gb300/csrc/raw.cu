// The raw-density entry point (Eq. 3.1's representation of the density: values on the grid,
// and inside each sphere its spherical-harmonic components on the logarithmic radial mesh).
// The caller gives the electron density at every node and each sphere's spherical component
// rho_00(r_j); the pseudo-density of Section 3 is built from the table, and the deposit
// replaces the spherical part inside each sphere by it (Section 1's monopole swap).
#include "internal.cuh"

namespace lasto {

namespace {

constexpr double RAW_PI = 3.14159265358979323846;

// One thread per sphere: q = sqrt(4pi) int_0^R rho_00 r^2 dr - Z (rule in ln r, rho_00
// constant on [0, r_min]), rho(R) = rho_00(R)/sqrt(4pi), rho'(R) from the one-sided fourth-
// order difference in ln r, and the quartic a + b r^2 + c r^4 meeting the three constraints
// (written out: c = (Q - rho R^3/3 + rho' R^4/15) 105/(8 R^7), b = rho'/(2R) - 2 c R^2,
// a = rho - rho' R/2 + c R^4 with Q = q/(4pi)).  Record: x y z R a b c h.  Also the
// geometry check: the sphere two nodes inside every face and disjoint from the others.
__global__ void k_raw_sphere_params(RawArgs a, double* __restrict__ rec, int* __restrict__ status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.na) return;
    const double Ri = a.R[i], rm = a.r_min;
    const int n = a.n_rad;
    const double h = log(Ri / rm) / (n - 1);
    const double* f = a.rho00 + (size_t)i * n;
    auto rr = [&](int j) { return j == n - 1 ? Ri : Ri * exp((j - (n - 1)) * h); };
    auto g = [&](int j) { const double x = rr(j); return f[j] * x * x * x; };
    double acc = f[0] * rm * rm * rm / 3.0;
    for (int j = 0; j + 1 < n; j++) {
        double w;
        if (j == 0) w = h / 24.0 * (9.0 * g(0) + 19.0 * g(1) - 5.0 * g(2) + g(3));
        else if (j == n - 2) w = h / 24.0 * (g(n - 4) - 5.0 * g(n - 3) + 19.0 * g(n - 2) + 9.0 * g(n - 1));
        else w = h / 24.0 * (-g(j - 1) + 13.0 * g(j) + 13.0 * g(j + 1) - g(j + 2));
        acc += w;
    }
    const double s4 = sqrt(4.0 * RAW_PI);
    const double q = s4 * acc - a.Z[i];
    const int m = n - 1;
    const double rho = f[m] / s4;
    const double drho = (25.0 * f[m] - 48.0 * f[m - 1] + 36.0 * f[m - 2] - 16.0 * f[m - 3] + 3.0 * f[m - 4]) /
                        (12.0 * h) / (Ri * s4);
    const double Q = q / (4.0 * RAW_PI), R2 = Ri * Ri, R4 = R2 * R2;
    const double c = (Q - rho * Ri * R2 / 3.0 + drho * R4 / 15.0) * 105.0 / (8.0 * R4 * R2 * Ri);
    const double b = drho / (2.0 * Ri) - 2.0 * c * R2;
    const double aa = rho - drho * Ri / 2.0 + c * R4;
    double* o = rec + (size_t)RAW_REC * i;
    o[0] = a.pos[3 * i];
    o[1] = a.pos[3 * i + 1];
    o[2] = a.pos[3 * i + 2];
    o[3] = Ri;
    o[4] = aa;
    o[5] = b;
    o[6] = c;
    o[7] = h;
    bool bad = false;
    for (int d = 0; d < 3; d++) {
        const double cc = a.pos[3 * i + d];
        if (!(cc - Ri >= a.ax[d][2] && cc + Ri <= a.ax[d][a.n[d] - 3])) bad = true;
    }
    for (int j = 0; j < a.na; j++) {
        if (j == i) continue;
        const double dx = a.pos[3 * i] - a.pos[3 * j], dy = a.pos[3 * i + 1] - a.pos[3 * j + 1],
                     dz = a.pos[3 * i + 2] - a.pos[3 * j + 2];
        if (sqrt(dx * dx + dy * dy + dz * dz) < Ri + a.R[j]) bad = true;
    }
    if (bad && status) atomicMax(status, (int)LASTO_ERR_GEOMETRY);
    if (!isfinite(q) || !isfinite(aa) || !isfinite(b) || !isfinite(c))
        if (status) atomicMax(status, (int)LASTO_ERR_NONFINITE);
}

// rho_00(r)/sqrt(4pi) of sphere i: cubic Lagrange in ln r on the four nearest samples; below
// r_min the straight line through the first two
__device__ __forceinline__ double monopole_at(const double* __restrict__ f, int n, double rm, double h, double r)
{
    if (r <= rm) {
        const double r1 = rm * exp(h);
        return f[0] + (f[1] - f[0]) * (r - rm) / (r1 - rm);
    }
    const double t = log(r / rm) / h;
    int j = (int)floor(t);
    j = j < 1 ? 1 : (j > n - 3 ? n - 3 : j);
    const double s = t - j;
    const double l0 = -s * (s - 1.0) * (s - 2.0) / 6.0, l1 = (s + 1.0) * (s - 1.0) * (s - 2.0) / 2.0;
    const double l2 = -(s + 1.0) * s * (s - 2.0) / 2.0, l3 = (s + 1.0) * s * (s - 1.0) / 6.0;
    return l0 * f[j - 1] + l1 * f[j] + l2 * f[j + 1] + l3 * f[j + 2];
}

// b = 4pi (ne - rho_00(r)/sqrt(4pi) + quartic(r)) inside sphere i (|x - X_i| < R_i), 4pi ne
// outside.  Ownership: an FP32 distance test decides all nodes farther than 1e-4 R^2 from
// a sphere surface; the rest are decided in FP64.
__global__ void __launch_bounds__(256) k_raw_deposit(RawArgs a, const double* __restrict__ rec,
                                                    double* __restrict__ b, int* __restrict__ owner,
                                                    int* __restrict__ status)
{
    // per atom, once per block: the FP32 position and the FP32 sphere-test bound (the node loop
    // then needs no FP64 conversion)
    extern __shared__ float4 raw_at[];
    for (int t = threadIdx.x; t < a.na; t += blockDim.x) {
        const double* o = rec + (size_t)RAW_REC * t;
        const float R2f = (float)(o[3] * o[3]);
        raw_at[t] = make_float4((float)o[0], (float)o[1], (float)o[2], R2f * (1.0f + 1e-4f));
    }
    __syncthreads();
    const unsigned N = (unsigned)a.n[0] * a.n[1] * a.n[2];   // < 2^31 (checked where grids are accepted)
    const unsigned P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= N) return;
    const unsigned nxy = (unsigned)a.n[0] * a.n[1];
    const int k = (int)(P / nxy), j = (int)((P - (unsigned)k * nxy) / a.n[0]), i = (int)(P - (unsigned)k * nxy - (unsigned)j * a.n[0]);
    const double x = a.ax[0][i], y = a.ax[1][j], z = a.ax[2][k];
    const float xf = (float)x, yf = (float)y, zf = (float)z;
    int own = -1;
    double r = 0.0;
    for (int t = 0; t < a.na; t++) {
        const float4 c = raw_at[t];
        const float dx = xf - c.x, dy = yf - c.y, dz = zf - c.z;
        const float r2f = dx * dx + dy * dy + dz * dz;
        if (r2f > c.w) continue;
        const double* o = rec + (size_t)RAW_REC * t;
        const double ex = x - o[0], ey = y - o[1], ez = z - o[2];
        const double d = sqrt(ex * ex + ey * ey + ez * ez);
        if (d < o[3]) {
            own = t;
            r = d;
            break;
        }
    }
    double v = a.ne[P];
    if (own >= 0) {
        const double* o = rec + (size_t)RAW_REC * own;
        const double rho0 = monopole_at(a.rho00 + (size_t)own * a.n_rad, a.n_rad, a.r_min, o[7], r) /
                            sqrt(4.0 * RAW_PI);
        v = v - rho0 + (o[4] + o[5] * r * r + o[6] * r * r * r * r);
    }
    const double bv = 4.0 * RAW_PI * v;
    b[P] = bv;
    if (owner) owner[P] = own;
    if (!isfinite(bv) && status) atomicMax(status, (int)LASTO_ERR_NONFINITE);
}

}  // namespace

cudaError_t launch_raw_sphere_params(const RawArgs& a, double* rec, int* status, cudaStream_t s)
{
    k_raw_sphere_params<<<(a.na + 63) / 64, 64, 0, s>>>(a, rec, status);
    return cudaGetLastError();
}

cudaError_t launch_raw_deposit(const RawArgs& a, const double* rec, double* b, int* owner, int* status, cudaStream_t s)
{
    const size_t N = (size_t)a.n[0] * a.n[1] * a.n[2];
    const size_t smem = sizeof(float4) * (size_t)a.na;
    if (smem > 200 * 1024 || N >= (size_t(1) << 31)) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_raw_deposit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_raw_deposit<<<(unsigned)((N + 255) / 256), 256, smem, s>>>(a, rec, b, owner, status);
    return cudaGetLastError();
}

}  // namespace lasto
