// Mesh axes, per-level operator / transfer tables and the exact coarse solve setup.
//
// Section 3 of the paper asks for fine meshes near the atoms and coarse meshes far
// away, with Dirichlet conditions at the edge of the finite domain, and a finite
// difference multigrid solve.  The graded tensor-product mesh below is the reading
// of that sentence; every multigrid level keeps every other node of the level above,
// and all stencil and transfer coefficients are tabulated per axis (O(n) data), so
// the smoother reads only u, b and (FP64) one inverse diagonal per node.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace lasto {

int set_cuda_error(Err* e, cudaError_t c, const char* what)
{
    if (e) {
        e->code = LASTO_ERR_CUDA;
        e->msg = std::string(what) + ": " + cudaGetErrorString(c);
    }
    return LASTO_ERR_CUDA;
}

int num_levels(const int n[3], int* coarse_n)
{
    int a = n[0], b = n[1], c = n[2], L = 1;
    while ((a > MAX_COARSE || b > MAX_COARSE || c > MAX_COARSE) && (a - 1) % 2 == 0 && (b - 1) % 2 == 0 &&
           (c - 1) % 2 == 0 && a >= 5 && b >= 5 && c >= 5) {
        a = (a + 1) / 2;
        b = (b + 1) / 2;
        c = (c + 1) / 2;
        L++;
    }
    if (a > MAX_COARSE || b > MAX_COARSE || c > MAX_COARSE) return -1;
    if (L > MAX_LEVELS) return -1;
    if (coarse_n) {
        coarse_n[0] = a;
        coarse_n[1] = b;
        coarse_n[2] = c;
    }
    return L;
}

// one axis: c + 7 FP64 tables of n (rw uses 3n) + 7 FP32 tables, in doubles
size_t axis_pool_doubles(int n) { return (size_t)n * (1 + 6 + 3) + ((size_t)n * (6 + 3) + 1) / 2 + 8; }

void carve_axis(AxisStore* a, int n, double* pool)
{
    a->n = n;
    double* p = pool;
    a->c = p; p += n;
    a->cm = p; p += n;
    a->cp = p; p += n;
    a->dg = p; p += n;
    a->dual = p; p += n;
    a->pl = p; p += n;
    a->pr = p; p += n;
    a->rw = p; p += 3 * (size_t)n;
    float* f = reinterpret_cast<float*>(p);
    a->cm32 = f; f += n;
    a->cp32 = f; f += n;
    a->dg32 = f; f += n;
    a->dual32 = f; f += n;
    a->pl32 = f; f += n;
    a->pr32 = f; f += n;
    a->rw32 = f; f += 3 * (size_t)n;
}

template <typename T>
static AxisT<T> axis_view(const AxisStore& a);
template <>
AxisT<double> axis_view<double>(const AxisStore& a)
{
    return AxisT<double>{a.c, a.cm, a.cp, a.dg, a.dual, a.pl, a.pr, a.rw, a.n};
}
template <>
AxisT<float> axis_view<float>(const AxisStore& a)
{
    return AxisT<float>{a.c, a.cm32, a.cp32, a.dg32, a.dual32, a.pl32, a.pr32, a.rw32, a.n};
}

LevelT<double> LevelStore::view64() const
{
    LevelT<double> v;
    for (int d = 0; d < 3; d++) v.ax[d] = axis_view<double>(ax[d]);
    v.inv_diag = inv_diag;
    set_dims(v, n[0], n[1], n[2]);
    return v;
}
LevelT<float> LevelStore::view32() const
{
    LevelT<float> v;
    for (int d = 0; d < 3; d++) v.ax[d] = axis_view<float>(ax[d]);
    v.inv_diag = nullptr;
    set_dims(v, n[0], n[1], n[2]);
    set_split(v, split32);
    return v;
}

// ---------------------------------------------------------------- mesh axis
__global__ void k_mesh_axis(int n, double c, double L, double A, double B, double p, double* x)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double m = 0.5 * (n - 1);
    const double xi = (i - m) / m;
    double v;
    if (i == 0) v = c - L;
    else if (i == n - 1) v = c + L;
    else {
        const double g = (B == 0.0) ? 0.0 : B * pow(fabs(xi), p);
        v = c + A * xi + copysign(g, xi);
    }
    x[i] = v;
}

__global__ void k_mesh_info(int n, double A, double B, double p, const double* x, double* info)
{
    const int m = (n - 1) / 2;
    info[0] = A;
    info[1] = B;
    info[2] = p;
    info[3] = x[m + 1] - x[m];
    info[4] = x[n - 1] - x[n - 2];
}

cudaError_t launch_mesh_axis(int n, double c, double L, double h_min, double h_max, double p_max, double* x,
                             double* info, cudaStream_t s)
{
    // grading parameters (host planning): slopes h_min m at the centre and h_max m at the ends
    const double m = 0.5 * (n - 1);
    double A = h_min * m, B = L - A, p = 1.0;
    if (B <= 1e-12 * L) {
        A = L;
        B = 0.0;
    } else {
        p = (h_max * m - A) / B;
        if (p > p_max) {
            p = p_max;
            B = (h_max * m - L) / (p_max - 1.0);
            A = L - B;
        }
    }
    k_mesh_axis<<<(n + 127) / 128, 128, 0, s>>>(n, c, L, A, B, p, x);
    if (info) k_mesh_info<<<1, 1, 0, s>>>(n, A, B, p, x, info);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- level tables
struct TabArgs {
    AxisStore ax[3];
    const double* src[3];
    int stride;
};

__global__ void k_level_tables(TabArgs a)
{
    const int d = blockIdx.y;
    const AxisStore& A = a.ax[d];
    const int n = A.n;
    const double* src = a.src[d];
    const int st = a.stride;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        auto C = [&](int t) { return src[(size_t)st * t]; };
        const double ci = C(i);
        A.c[i] = ci;
        double cm = 0.0, cp = 0.0, dual, pl = 1.0, pr = 0.0;
        if (i > 0 && i < n - 1) {
            const double hm = ci - C(i - 1), hp = C(i + 1) - ci;
            cm = 2.0 / ((hm + hp) * hm);
            cp = 2.0 / ((hm + hp) * hp);
            dual = 0.5 * (hm + hp);
            if (i & 1) {
                pl = hp / (hm + hp);
                pr = hm / (hm + hp);
            }
        } else {
            dual = (i == 0) ? 0.5 * (C(1) - ci) : 0.5 * (ci - C(n - 2));
        }
        A.cm[i] = cm;
        A.cp[i] = cp;
        A.dg[i] = cm + cp;
        A.dual[i] = dual;
        A.pl[i] = pl;
        A.pr[i] = pr;
        A.cm32[i] = (float)cm;
        A.cp32[i] = (float)cp;
        A.dg32[i] = (float)(cm + cp);
        A.dual32[i] = (float)dual;
        A.pl32[i] = (float)pl;
        A.pr32[i] = (float)pr;
        // restriction weights of coarse node I = i on the next level (nc = (n+1)/2)
        const int nc = (n + 1) / 2;
        double w0 = 0.0, w1 = 0.0, w2 = 0.0;
        if ((n - 1) % 2 == 0 && i >= 1 && i <= nc - 2) {
            const int f = 2 * i;
            const double Vc = 0.5 * (C(f + 2) - C(f - 2));
            const double hm1 = C(f - 1) - C(f - 2), hp1 = C(f) - C(f - 1);     // fine node f-1 (odd)
            const double hm3 = C(f + 1) - C(f), hp3 = C(f + 2) - C(f + 1);     // fine node f+1 (odd)
            const double v1 = 0.5 * (hm1 + hp1), v2 = 0.5 * (hp1 + hm3), v3 = 0.5 * (hm3 + hp3);
            w0 = (hm1 / (hm1 + hp1)) * v1 / Vc;   // weight of coarse node I at fine f-1 (its right end)
            w1 = v2 / Vc;
            w2 = (hp3 / (hm3 + hp3)) * v3 / Vc;   // weight of coarse node I at fine f+1 (its left end)
        }
        A.rw[3 * i] = w0;
        A.rw[3 * i + 1] = w1;
        A.rw[3 * i + 2] = w2;
        A.rw32[3 * i] = (float)w0;
        A.rw32[3 * i + 1] = (float)w1;
        A.rw32[3 * i + 2] = (float)w2;
    }
}

cudaError_t launch_level_tables(const LevelStore& lv, const LevelStore* /*coarse*/, const double* src_coords[3],
                                int src_stride, cudaStream_t s)
{
    TabArgs a;
    for (int d = 0; d < 3; d++) {
        a.ax[d] = lv.ax[d];
        a.src[d] = src_coords[d];
    }
    a.stride = src_stride;
    const int nmax = std::max(lv.n[0], std::max(lv.n[1], lv.n[2]));
    k_level_tables<<<dim3((nmax + 127) / 128, 3), 128, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- inverse diagonal
__global__ void k_inv_diag(LevelT<double> L, double* inv)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= L.nx) return;
    const size_t P = ((size_t)k * L.ny + j) * L.nx + i;
    const bool face = i == 0 || j == 0 || k == 0 || i == L.nx - 1 || j == L.ny - 1 || k == L.nz - 1;
    inv[P] = face ? 0.0 : -1.0 / (L.ax[0].dg[i] + L.ax[1].dg[j] + L.ax[2].dg[k]);
}

cudaError_t launch_inv_diag(const LevelStore& lv, cudaStream_t s)
{
    LevelT<double> L = lv.view64();
    k_inv_diag<<<dim3((L.nx + 127) / 128, L.ny, L.nz), 128, 0, s>>>(L, lv.inv_diag);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- coarse fast diagonalisation
// The 1-D operator T (interior rows: cm, -(cm+cp), cp) is similar to the symmetric
// S = V^{1/2} T V^{-1/2} (V = dual lengths), whose off-diagonal is sqrt(cp_i cm_{i+1}).
// Cyclic Jacobi rotations (Golub & Van Loan, symmetric Schur decomposition) give
// S = Q diag(lam) Q^T, so A^{-1} = (x) V^{-1/2} Q  diag(1/(lx+ly+lz))  (x) Q^T V^{1/2}.
// One warp per axis; a rotation's row and column updates run across the lanes (lane k owns
// element k), each element computed exactly as in the sequential sweep.
__global__ void __launch_bounds__(96) k_coarse_eig(AxisStore ax0, AxisStore ax1, AxisStore ax2, CoarseEig* out)
{
    constexpr int MM = MAX_COARSE - 2;
    __shared__ double Ssh[3][MM][MM], Qsh[3][MM][MM];
    const int d = threadIdx.x >> 5, k = threadIdx.x & 31;
    const AxisStore& A = d == 0 ? ax0 : d == 1 ? ax1 : ax2;
    const int m = A.n - 2;
    double(*S)[MM] = Ssh[d];
    double(*Q)[MM] = Qsh[d];
    if (k < m) {
        for (int j = 0; j < m; j++) {
            S[k][j] = 0.0;
            Q[k][j] = (k == j) ? 1.0 : 0.0;
        }
    }
    __syncwarp();
    if (k < m) {
        S[k][k] = -A.dg[k + 1];
        if (k + 1 < m) S[k][k + 1] = S[k + 1][k] = sqrt(A.cp[k + 1] * A.cm[k + 2]);
    }
    __syncwarp();
    int ok = 0;
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0, dia = 0.0;
        for (int p = 0; p < m; p++) {
            dia += S[p][p] * S[p][p];
            for (int q = p + 1; q < m; q++) off += S[p][q] * S[p][q];
        }
        if (off <= 1e-32 * dia) {
            ok = 1;
            break;
        }
        for (int p = 0; p < m; p++)
            for (int q = p + 1; q < m; q++) {
                const double spq = S[p][q];
                if (spq == 0.0) continue;
                const double tau = (S[q][q] - S[p][p]) / (2.0 * spq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                __syncwarp();
                if (k < m) {
                    const double kp = S[k][p], kq = S[k][q];
                    S[k][p] = c * kp - s * kq;
                    S[k][q] = s * kp + c * kq;
                }
                __syncwarp();
                if (k < m) {
                    const double pk = S[p][k], qk = S[q][k];
                    S[p][k] = c * pk - s * qk;
                    S[q][k] = s * pk + c * qk;
                    const double qp = Q[k][p], qq = Q[k][q];
                    Q[k][p] = c * qp - s * qq;
                    Q[k][q] = s * qp + c * qq;
                }
                __syncwarp();
            }
    }
    if (k == 0) {
        out->m[d] = m;
        out->ok[d] = ok;
    }
    for (int p = 0; p < m; p++) {
        if (k == 0) out->lam[d][p] = S[p][p];
        if (k < m) {
            const double sv = sqrt(A.dual[k + 1]);
            out->F[d][p * m + k] = Q[k][p] * sv;
            out->B[d][k * m + p] = Q[k][p] / sv;
        }
    }
}

cudaError_t launch_coarse_eig(const LevelStore& L, CoarseEig* eig, cudaStream_t s)
{
    k_coarse_eig<<<1, 96, 0, s>>>(L.ax[0], L.ax[1], L.ax[2], eig);
    return cudaGetLastError();
}

}  // namespace lasto
