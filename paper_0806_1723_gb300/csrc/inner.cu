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
// x = ln r with the cubic through the four nearest samples per interval.  The density
// projection runs its Slater sums in FP32 pairs; the radial solve is one block per (atom, LM)
// with the interval integrals summed as block-wide prefix (I1) and suffix (I2) scans.
#include <cmath>

#include "df.cuh"
#include "internal.cuh"

namespace lasto {

namespace {

constexpr int SD_NT = 128;
constexpr int SD_MAXQ = 2048;      // quadrature points per sphere
constexpr double SD_EXP_CUT = 40.0;
constexpr float SD_FAR = 20.0f;   // Slater terms beyond zeta r = 20 in plain FP32

using dfa::df;

struct SdExp {
    float h[64], l[64];   // 2^(-j/64) as double-floats
};

// rho_LM(r_j) of atom a = blockIdx.y at radius j = blockIdx.x.  rec: sphere records
// (position, radius, Slater weights and exponents per atom); quad [nq][28]: unit vector and
// w_q S_lm(u_q).  The Slater sum at each quadrature point runs in FP32 pairs (about 44 bits:
// Tang's table-driven exp), with positions taken relative to the sphere's centre so that the
// pairs stay small; terms beyond zeta r = 20 (below e^-20 of their weight) in plain FP32.  The
// projection sums over the quadrature points are FP64.
__global__ void __launch_bounds__(SD_NT) k_sphere_density(int na, const double* __restrict__ rec,
                                                          const double* __restrict__ clm,
                                                          const double* __restrict__ quad, int nq, int n_rad,
                                                          double r_min, SdExp tab, double* __restrict__ out)
{
    extern __shared__ float sd_sm[];   // per atom: D = pos_t - pos_a (3 pairs), W (3 pairs)
    __shared__ double rq[SD_MAXQ];     // the density at the quadrature points
    __shared__ double cs[NLM];         // own nonspherical part: prefactor(r) c_lm (r/R)^l
    const int a = blockIdx.y, j = blockIdx.x, tid = threadIdx.x;
    const double* ra = rec + (size_t)SPHERE_REC_DOUBLES * a;
    const double Ra = ra[3];
    const double dx = log(Ra / r_min) / (n_rad - 1);
    const double r = (j == n_rad - 1) ? Ra : Ra * exp((j - (n_rad - 1)) * dx);
    // own nonspherical part zeta_1^3/(8 pi) e^{-zeta_1 r} (1 - r^2/R^2)^2 sum c_lm (r/R)^l y_lm:
    // everything but y_lm depends on the radius only, once per block
    if (tid < NLM) {
        double v = 0.0;
        if (tid > 0 && r < Ra) {
            const double z1 = ra[7], sr = r / Ra, tt = 1.0 - sr * sr;
            const int l = tid >= 16 ? 4 : tid >= 9 ? 3 : tid >= 4 ? 2 : 1;
            double sl = sr;
            for (int p = 1; p < l; p++) sl *= sr;
            v = z1 * z1 * z1 / (8.0 * 3.14159265358979323846) * exp(-z1 * r) * tt * tt * clm[24 * (size_t)a + tid - 1] * sl;
        }
        cs[tid] = v;
    }
    for (int t = tid; t < na; t += SD_NT) {
        const double* rt = rec + (size_t)SPHERE_REC_DOUBLES * t;
        float* o = sd_sm + 12 * t;
        for (int c = 0; c < 3; c++) {
            const df D = dfa::from_double(rt[c] - ra[c]);
            o[2 * c] = D.h;
            o[2 * c + 1] = D.l;
            const df W = dfa::from_double(rt[4 + c]);
            o[6 + 2 * c] = W.h;
            o[7 + 2 * c] = W.l;
        }
    }
    __syncthreads();
    // the exponents are the same on every atom (checked by the sphere kernel)
    df zt[3];
    float zmin = 1e30f;
    for (int c = 0; c < 3; c++) {
        zt[c] = dfa::from_double(ra[7 + c]);
        zmin = fminf(zmin, zt[c].h);
    }
    const float cut = (float)SD_EXP_CUT / zmin, cut2 = cut * cut * (1.0f + 1e-5f);
    bool twice[3];   // zeta_c exactly twice zeta_0
#pragma unroll
    for (int c = 0; c < 3; c++) twice[c] = c > 0 && zt[c].h == 2.0f * zt[0].h && zt[c].l == 2.0f * zt[0].l;
    const float far = SD_FAR / zmin, far2 = far * far * (1.0f + 1e-4f);
    const double y00 = 0.28209479177387814;   // S_00 = 1 / (2 sqrt(pi)); quad[3] = w_q S_00
    for (int q = tid; q < nq; q += SD_NT) {
        const double* Q = quad + 28 * (size_t)q;
        const df px = dfa::from_double(r * Q[0]), py = dfa::from_double(r * Q[1]), pz = dfa::from_double(r * Q[2]);
        df rho = {0.0f, 0.0f};
        float rfar = 0.0f;   // the terms beyond zeta d = SD_FAR in plain FP32, added once below
        for (int t = 0; t < na; t++) {
            const float* o = sd_sm + 12 * t;
            const float fx = (px.h - o[0]) + (px.l - o[1]), fy = (py.h - o[2]) + (py.l - o[3]);
            const float fz = (pz.h - o[4]) + (pz.l - o[5]);
            const float r2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
            if (r2f > cut2) continue;
            if (r2f > far2) {
                const float rf = sqrtf(r2f);
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const float e = zt[c].h * rf;
                    if (e < (float)SD_EXP_CUT) rfar = fmaf(o[6 + 2 * c], expf(-e), rfar);
                }
                continue;
            }
            const df ex = dfa::add(px, df{-o[0], -o[1]});
            const df ey = dfa::add(py, df{-o[2], -o[3]});
            const df ez = dfa::add(pz, df{-o[4], -o[5]});
            const df d2 = dfa::add(dfa::add(dfa::sqr(ex), dfa::sqr(ey)), dfa::sqr(ez));
            const df d = dfa::sqrt_df(d2);
            df e0 = {0.0f, 0.0f};
            bool have0 = false;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const df e = dfa::mul(d, zt[c]);
                if (e.h >= (float)SD_EXP_CUT) continue;
                if (e.h > SD_FAR) {
                    rfar = fmaf(o[6 + 2 * c], expf(-e.h), rfar);
                } else {
                    // zeta_c = 2 zeta_0: e^{-zeta_c d} = (e^{-zeta_0 d})^2
                    const df ec = (c > 0 && twice[c] && have0) ? dfa::sqr(e0) : dfa::exp_neg(e, tab.h, tab.l);
                    if (c == 0) {
                        e0 = ec;
                        have0 = true;
                    }
                    rho = dfa::add(rho, dfa::mul(df{o[6 + 2 * c], o[7 + 2 * c]}, ec));
                }
            }
        }
        double rhod = dfa::to_double(dfa::add_f(rho, rfar));
        if (r < Ra) {
            // quad[4..] = w_q y_lm(q): one division by w_q = quad[3] / y_00 per point
            double ang = 0.0;
            for (int lm = 1; lm < NLM; lm++) ang = fma(cs[lm], Q[3 + lm], ang);
            rhod += ang * (y00 / Q[3]);
        }
        rq[q] = rhod;
    }
    __syncthreads();
    // the projection: warp w takes lm = w, w + 4, ...; lanes split the quadrature points
    const int lane = tid & 31, w = tid >> 5;
    for (int lm = w; lm < NLM; lm += SD_NT / 32) {
        double acc = 0.0;
        for (int q = lane; q < nq; q += 32) acc = fma(quad[28 * (size_t)q + 3 + lm], rq[q], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) out[((size_t)a * NLM + lm) * n_rad + j] = acc;
    }
}

__device__ __forceinline__ double seg_integral(double g0, double g1, double g2, double g3, int kind, double h)
{
    // kind 0: first interval (samples j..j+3), 1: interior (j-1..j+2), 2: last (j-2..j+1)
    if (kind == 0) return h / 24.0 * (9.0 * g0 + 19.0 * g1 - 5.0 * g2 + g3);
    if (kind == 2) return h / 24.0 * (g0 - 5.0 * g1 + 19.0 * g2 + 9.0 * g3);
    return h / 24.0 * (-g0 + 13.0 * g1 + 13.0 * g2 - g3);
}

constexpr int IS_NT = 128;
constexpr int IS_MAX = 4096;   // radial points per sphere

// inclusive scan of one double per thread over the block (warp shuffles, then the warps' totals)
__device__ __forceinline__ double block_incl_scan(double v, double* wsum)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    __syncthreads();
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    for (int q = 0; q < w; q++) v += wsum[q];
    return v;
}

// One block per (atom, lm).  The integrands at the mesh points, the cubic-rule integral over
// each interval, then I1 as a prefix sum and I2 as a suffix sum of the intervals (each thread
// a contiguous run of intervals, the runs' totals scanned across the block), then V_LM.
__global__ void __launch_bounds__(IS_NT) k_inner_solve(int na, const double* __restrict__ R,
                                                       const double* __restrict__ Z, int n, double r_min,
                                                       const double* __restrict__ rho_lm,
                                                       const double* __restrict__ vR, double* __restrict__ v)
{
    extern __shared__ double is_sm[];   // x[n], g1[n], g2[n], seg1[n], seg2[n]
    __shared__ double wsum[IS_NT / 32];
    double* xs = is_sm;
    double* g1 = xs + n;
    double* g2 = g1 + n;
    double* s1 = g2 + n;
    double* s2 = s1 + n;
    const int t = blockIdx.x, a = t / NLM, lm = t % NLM, L = l_of_lm(lm);
    const double Ra = R[a];
    const double h = log(Ra / r_min) / (n - 1);
    const double* rho = rho_lm + (size_t)t * n;
    double* out = v + (size_t)t * n;
    for (int j = threadIdx.x; j < n; j += IS_NT) {
        const double x = j == n - 1 ? Ra : Ra * exp((j - (n - 1)) * h);
        double xl = 1.0;
        for (int e = 0; e < L; e++) xl *= x;
        xs[j] = x;
        g1[j] = rho[j] * xl * x * x * x;   // rho r^(L+2) dr = rho r^(L+3) d(ln r)
        g2[j] = rho[j] * x * x / xl;       // rho r^(1-L) dr = rho r^(2-L) d(ln r)
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n - 1; j += IS_NT) {
        const int b = j == 0 ? 0 : (j == n - 2 ? n - 4 : j - 1);
        const int kind = j == 0 ? 0 : (j == n - 2 ? 2 : 1);
        s1[j] = seg_integral(g1[b], g1[b + 1], g1[b + 2], g1[b + 3], kind, h);
        s2[j] = seg_integral(g2[b], g2[b + 1], g2[b + 2], g2[b + 3], kind, h);
    }
    __syncthreads();
    // contiguous runs of intervals per thread: [c0, c1)
    const int m = n - 1, per = (m + IS_NT - 1) / IS_NT;
    const int c0 = min(m, (int)threadIdx.x * per), c1 = min(m, c0 + per);
    double run1 = 0.0, run2 = 0.0;
    for (int j = c0; j < c1; j++) {
        run1 += s1[j];
        run2 += s2[j];
    }
    const double inc1 = block_incl_scan(run1, wsum);
    __syncthreads();
    const double inc2 = block_incl_scan(run2, wsum);
    __syncthreads();
    if (threadIdx.x == IS_NT - 1) {
        wsum[0] = inc1;   // I1 over all intervals
        wsum[1] = inc2;   // I2 over all intervals
    }
    __syncthreads();
    const double tot1 = wsum[0], tot2 = wsum[1];
    const double I1_0 = g1[0] / (L + 3);   // rho taken constant on [0, r_0]: rho_0 r_0^(L+3) / (L+3)
    const double vr = vR[(size_t)a * NLM + lm];
    const double c = 4.0 * 3.14159265358979323846 / (2 * L + 1);
    const double sq4pi = 3.5449077018110318;
    double RaL = 1.0;
    for (int e = 0; e < L; e++) RaL *= Ra;
    const double R2L1 = RaL * RaL * Ra;
    const double I1R = I1_0 + tot1;
    // points [c0, c1) of this thread's run, and the last point m with the run that ends there:
    // I1 at point j = I1_0 + intervals [0, j), I2 = intervals [j, m)
    if (c0 < c1) {
        double p1 = inc1 - run1, p2 = tot2 - (inc2 - run2);
        const int last = c1 == m ? m : c1 - 1;
        for (int j = c0; j <= last; j++) {
            if (j > c0) {
                p1 += s1[j - 1];
                p2 -= s2[j - 1];
            }
            const double x = xs[j];
            double xl = 1.0;
            for (int e = 0; e < L; e++) xl *= x;
            const double I1 = I1_0 + p1;
            const double I2 = j == m ? 0.0 : p2;
            double val = vr * (xl / RaL) - c * (I1 / (xl * x) + xl * I2 - xl * I1R / R2L1);
            if (L == 0) val += sq4pi * Z[a] * (1.0 / x - 1.0 / Ra);
            out[j] = val;
        }
    }
}

}  // namespace

cudaError_t launch_sphere_density(int na, const double* rec, const double* clm, const double* quad, int nq,
                                  int n_rad, double r_min, double* out, cudaStream_t s)
{
    SdExp tab;
    for (int q = 0; q < 64; q++) {
        const double v = std::exp2(-q / 64.0);
        tab.h[q] = (float)v;
        tab.l[q] = (float)(v - (double)tab.h[q]);
    }
    const size_t smem = sizeof(float) * 12 * (size_t)na;
    if (smem > 160 * 1024 || nq > SD_MAXQ) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_sphere_density, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    k_sphere_density<<<dim3((unsigned)n_rad, (unsigned)na), SD_NT, smem, s>>>(na, rec, clm, quad, nq, n_rad, r_min,
                                                                              tab, out);
    return cudaGetLastError();
}

cudaError_t launch_inner_solve(int na, const double* R, const double* Z, int n_rad, double r_min,
                               const double* rho_lm, const double* vR, double* v, cudaStream_t s)
{
    if (n_rad > IS_MAX) return cudaErrorInvalidValue;
    const size_t smem = sizeof(double) * 5 * (size_t)n_rad;
    cudaError_t e = cudaFuncSetAttribute(k_inner_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(double) * 5 * IS_MAX));
    if (e != cudaSuccess) return e;
    k_inner_solve<<<(unsigned)(na * NLM), IS_NT, smem, s>>>(na, R, Z, n_rad, r_min, rho_lm, vR, v);
    return cudaGetLastError();
}

}  // namespace lasto
