// Inside the atom spheres (Section 3, Eq. 3.4-3.7): the density's spherical-harmonic
// components on a logarithmic radial mesh, and the inner Dirichlet problem whose boundary
// values are the sphere-surface coefficients V_LM(R) of the interstitial solve.
//
// Radial mesh of sphere a: r_j = R_a exp((j - (n-1)) dx), dx = ln(R_a / r_min) / (n - 1); the
// paper uses a logarithmic mesh of 429 points.  rho_LM(r_j) is Eq. 3.7's surface projection
// taken on the sphere of radius r_j (the projection's Gauss-Legendre x uniform rule).  The
// inner solve is the Green's-function form of Eq. 3.5 with the overall sign that satisfies
// Eq. 3.4 (d2/dr2 + 2/r d/dr - L(L+1)/r^2) V_LM = 4pi (rho_LM - delta_L0 Z delta):
//   V_LM(r) = V_LM(R) (r/R)^L - 4pi/(2L+1) [ r^-(L+1) I1(r) + r^L I2(r) - r^L R^-(2L+1) I1(R) ]
//           + delta_L0 sqrt(4pi) Z (1/r - 1/R),
// I1(r) = int_0^r rho_LM r'^(L+2) dr', I2(r) = int_r^R rho_LM r'^(1-L) dr', integrated in
// x = ln r with the cubic through the four nearest samples per interval.
#include "internal.cuh"

namespace lasto {

namespace {

constexpr int SD_NT = 128;
constexpr double SD_EXP_CUT = 40.0;
constexpr double SD_FAR = 20.0;   // Slater terms beyond zeta r = 20 in plain FP32

// rho_LM(r_j) of atom a = blockIdx.y at radius j = blockIdx.x.  rec: sphere records
// (position, radius, Slater weights and exponents per atom); quad [nq][28]: unit vector and
// w_q S_lm(u_q).
__global__ void __launch_bounds__(SD_NT) k_sphere_density(int na, const double* __restrict__ rec,
                                                          const double* __restrict__ clm,
                                                          const double* __restrict__ quad, int nq, int n_rad,
                                                          double r_min, double* __restrict__ out)
{
    __shared__ double red[NLM][SD_NT];
    const int a = blockIdx.y, j = blockIdx.x, tid = threadIdx.x;
    const double* ra = rec + (size_t)SPHERE_REC_DOUBLES * a;
    const double Ra = ra[3];
    const double dx = log(Ra / r_min) / (n_rad - 1);
    const double r = (j == n_rad - 1) ? Ra : Ra * exp((j - (n_rad - 1)) * dx);
    const double y00 = 0.28209479177387814;   // S_00 = 1 / (2 sqrt(pi)); quad[3] = w_q S_00
    double acc[NLM];
#pragma unroll
    for (int lm = 0; lm < NLM; lm++) acc[lm] = 0.0;
    for (int q = tid; q < nq; q += SD_NT) {
        const double* Q = quad + 28 * (size_t)q;
        const double px = ra[0] + r * Q[0], py = ra[1] + r * Q[1], pz = ra[2] + r * Q[2];
        double rho = 0.0;
        for (int t = 0; t < na; t++) {
            const double* rt = rec + (size_t)SPHERE_REC_DOUBLES * t;
            const double ex = px - rt[0], ey = py - rt[1], ez = pz - rt[2];
            const double d = sqrt(ex * ex + ey * ey + ez * ez);
            for (int k = 0; k < 3; k++) {
                const double e = rt[7 + k] * d;
                if (e >= SD_EXP_CUT) continue;
                rho += (e > SD_FAR) ? (double)((float)rt[4 + k] * expf(-(float)e)) : rt[4 + k] * exp(-e);
            }
        }
        // own nonspherical part: zeta_1^3/(8 pi) e^{-zeta_1 r} (1 - r^2/R^2)^2 sum c_lm (r/R)^l y_lm
        if (r < Ra) {
            const double z1 = ra[7], w = Q[3] / y00, s = r / Ra, tt = 1.0 - s * s;
            double ang = 0.0, sl = s;
            for (int lm = 1; lm < NLM; lm++) {
                if (lm == 4 || lm == 9 || lm == 16) sl *= s;
                ang += clm[24 * (size_t)a + lm - 1] * sl * (Q[3 + lm] / w);
            }
            rho += z1 * z1 * z1 / (8.0 * 3.14159265358979323846) * exp(-z1 * r) * tt * tt * ang;
        }
#pragma unroll
        for (int lm = 0; lm < NLM; lm++) acc[lm] = fma(Q[3 + lm], rho, acc[lm]);
    }
#pragma unroll
    for (int lm = 0; lm < NLM; lm++) red[lm][tid] = acc[lm];
    __syncthreads();
    for (int st = SD_NT / 2; st > 0; st >>= 1) {
        if (tid < st)
            for (int lm = 0; lm < NLM; lm++) red[lm][tid] += red[lm][tid + st];
        __syncthreads();
    }
    if (tid < NLM) out[((size_t)a * NLM + tid) * n_rad + j] = red[tid][0];
}

__device__ __forceinline__ double seg_integral(double g0, double g1, double g2, double g3, int kind, double h)
{
    // kind 0: first interval (samples j..j+3), 1: interior (j-1..j+2), 2: last (j-2..j+1)
    if (kind == 0) return h / 24.0 * (9.0 * g0 + 19.0 * g1 - 5.0 * g2 + g3);
    if (kind == 2) return h / 24.0 * (g0 - 5.0 * g1 + 19.0 * g2 + 9.0 * g3);
    return h / 24.0 * (-g0 + 13.0 * g1 + 13.0 * g2 - g3);
}

// One thread per (atom, lm).  The forward integral I1 is parked in v, then the backward pass
// forms I2 and overwrites v with V_LM.
__global__ void k_inner_solve(int na, const double* __restrict__ R, const double* __restrict__ Z, int n,
                              double r_min, const double* __restrict__ rho_lm, const double* __restrict__ vR,
                              double* __restrict__ v)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= na * NLM) return;
    const int a = t / NLM, lm = t % NLM, L = l_of_lm(lm);
    const double Ra = R[a];
    const double h = log(Ra / r_min) / (n - 1);
    const double* rho = rho_lm + (size_t)t * n;
    double* out = v + (size_t)t * n;
    auto rr = [&](int j) { return j == n - 1 ? Ra : Ra * exp((j - (n - 1)) * h); };
    auto g1 = [&](int j) { const double x = rr(j); return rho[j] * pow(x, L + 2) * x; };
    auto g2 = [&](int j) { const double x = rr(j); return rho[j] * pow(x, 1 - L) * x; };
    auto seg = [&](auto g, int j) {
        if (j == 0) return seg_integral(g(0), g(1), g(2), g(3), 0, h);
        if (j == n - 2) return seg_integral(g(n - 4), g(n - 3), g(n - 2), g(n - 1), 2, h);
        return seg_integral(g(j - 1), g(j), g(j + 1), g(j + 2), 1, h);
    };
    double I1 = rho[0] * pow(rr(0), L + 3) / (L + 3);
    out[0] = I1;
    for (int j = 0; j + 1 < n; j++) {
        I1 += seg(g1, j);
        out[j + 1] = I1;
    }
    const double I1R = I1, vr = vR[(size_t)a * NLM + lm];
    const double c = 4.0 * 3.14159265358979323846 / (2 * L + 1);
    const double sq4pi = 3.5449077018110318;
    double I2 = 0.0;
    for (int j = n - 1; j >= 0; j--) {
        if (j < n - 1) I2 += seg(g2, j);
        const double x = rr(j), rl = pow(x, L);
        double val = vr * pow(x / Ra, L) - c * (out[j] / pow(x, L + 1) + rl * I2 - rl * I1R / pow(Ra, 2 * L + 1));
        if (L == 0) val += sq4pi * Z[a] * (1.0 / x - 1.0 / Ra);
        out[j] = val;
    }
}

}  // namespace

cudaError_t launch_sphere_density(int na, const double* rec, const double* clm, const double* quad, int nq,
                                  int n_rad, double r_min, double* out, cudaStream_t s)
{
    k_sphere_density<<<dim3((unsigned)n_rad, (unsigned)na), SD_NT, 0, s>>>(na, rec, clm, quad, nq, n_rad, r_min,
                                                                           out);
    return cudaGetLastError();
}

cudaError_t launch_inner_solve(int na, const double* R, const double* Z, int n_rad, double r_min,
                               const double* rho_lm, const double* vR, double* v, cudaStream_t s)
{
    const int total = na * NLM;
    k_inner_solve<<<(total + 127) / 128, 128, 0, s>>>(na, R, Z, n_rad, r_min, rho_lm, vR, v);
    return cudaGetLastError();
}

}  // namespace lasto
