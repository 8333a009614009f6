// Allocation-free variant of the density deposit.
//
// lasto_op_deposit takes a few hundred bytes per atom of device scratch (the per-sphere
// pseudo-density records) from the stream-ordered allocator.  Some callers cannot
// allocate device memory at the point where they need a deposit: code that runs under
// a fixed memory budget set at start-up, programs whose device heap is owned by another
// framework's caching allocator, and real-time loops that forbid allocation after
// initialisation.  This file gives them the same kernels with the records in one
// fixed, file-scope device array instead.
#include <mutex>

#include "internal.cuh"

namespace {

// Largest cluster the allocation-free deposit accepts.  The array below is
// LASTO_NOALLOC_MAX_ATOMS * 48 doubles = 384 KiB, held by every device that loads the
// library until the process exits.
constexpr int LASTO_NOALLOC_MAX_ATOMS = 1024;

static __device__ __align__(256) double g_sphere_records[LASTO_NOALLOC_MAX_ATOMS * lasto::SPHERE_REC_DOUBLES];

constexpr int MAX_DEVICES = 64;
double* g_records_addr[MAX_DEVICES] = {nullptr};
std::mutex g_setup_mutex;

// Device address of g_sphere_records on the current device (the host-side symbol is not
// a device address).  Looked up once per device, with that device current.
int records_address(double** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return LASTO_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_records_addr[dev]) {
        lasto::init_device_constants();
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_sphere_records);
        if (e != cudaSuccess || !p) return LASTO_ERR_CUDA;
        g_records_addr[dev] = static_cast<double*>(p);
    }
    *out = g_records_addr[dev];
    return LASTO_OK;
}

}  // namespace

extern "C" int lasto_op_deposit_noalloc(const lasto_cluster* cl, int precision, double* b, int* owner, int* status,
                                        void* stream)
{
    // the same grid checks as lasto_op_deposit, then the array's atom limit
    if (!cl || !b || cl->n_atoms < 1 || !lasto::op_grid_ok(cl->n, cl->x, cl->y, cl->z)) return LASTO_ERR_INVALID_ARG;
    if (cl->n_atoms > LASTO_NOALLOC_MAX_ATOMS) return LASTO_ERR_INVALID_ARG;
    if (precision != LASTO_PREC_FP64 && precision != LASTO_PREC_MIXED) return LASTO_ERR_INVALID_ARG;
    double* rec = nullptr;
    const int st = records_address(&rec);
    if (st != LASTO_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the sphere kernel writes every record the deposit reads, so nothing needs clearing
    cudaError_t e = lasto::launch_sphere_params(*cl, cl->x, cl->y, cl->z, rec, nullptr, nullptr, nullptr, nullptr,
                                                status, s);
    if (e == cudaSuccess) e = lasto::launch_deposit(*cl, rec, precision, b, owner, nullptr, nullptr, status, s);
    return lasto::op_status(e);
}
