// jfnk_residual_noalloc: the residual R(u) evaluated without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a residual: code that
// runs while a CUDA stream is being captured into a graph (cudaMalloc is not allowed during
// capture), code in processes where another framework's pool owns the device memory, and
// latency-sensitive loops that must not take the implicit device synchronisation of
// cudaMalloc/cudaFree.  For them this entry point takes its scratch (the caller-order to
// internal-order copies of u and R, the cell gradients, the neo-Hookean traction operators
// and the two face-flux arrays) from one file-scope device array of fixed size instead of
// the context's buffers.  The caller still passes u and R.
//
// Properties a caller must know:
//  * the array holds kNoallocScratchDoubles doubles (16 MiB) and stays resident on every GPU
//    that loads the library, until the process exits;
//  * all calls share it and it keeps the contents of the last call; every element a call
//    reads it first writes, so nothing needs clearing between calls;
//  * calls whose work overlaps on the GPU (different streams, or several contexts on one
//    device) race on the array: serialise them;
//  * the first call on a device looks up the array's device address (cudaGetSymbolAddress)
//    with that device current; make that first call before any stream capture.
#include <mutex>

#include "jfnk_internal.h"

namespace {

constexpr size_t kNoallocScratchDoubles = size_t(1) << 21;  // 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

std::mutex g_addr_mutex;
double* g_addr[kMaxDevices] = {nullptr};

// device address of the scratch array for `device` (which must be current); nullptr on error
double* scratch_address(int device, cudaError_t* err)
{
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    *err = cudaSuccess;
    if (device < 0 || device >= kMaxDevices) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    if (!g_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            *err = e;
            return nullptr;
        }
        g_addr[device] = (double*)p;
    }
    return g_addr[device];
}

}  // namespace

extern "C" int jfnk_residual_noalloc(jfnk_ctx* c, const double* u, double* R, void* stream)
{
    if (!c || !u || !R) return JFNK_EINVAL;
    if (c->dirty || !c->gdev)
        return jfnk_fail(c, JFNK_ESTATE, "jfnk_residual_noalloc: call jfnk_setup() first (this entry point never allocates)");
    const jfnk::DevMesh& m = c->dm;
    const size_t nc = (size_t)m.nc;
    const size_t need = 3 * nc + 9 * nc + (c->law_mode != 0 ? 9 * nc : 0) + 3 * (size_t)m.nflux +
                        3 * (size_t)m.ni + 3 * nc;
    if (need > kNoallocScratchDoubles)
        return jfnk_fail(c, JFNK_EINVAL,
                         "jfnk_residual_noalloc: the mesh needs " + std::to_string(need) + " scratch doubles, more than the " +
                             std::to_string(kNoallocScratchDoubles) + " of the fixed array (use jfnk_residual)");
    if (cudaSetDevice(c->opt.device) != cudaSuccess) return jfnk_cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaError_t e;
    double* base = scratch_address(c->opt.device, &e);
    if (!base) return jfnk_cuda_fail(c, e, "cudaGetSymbolAddress");
    int rc = jfnk_use_stream(c, (cudaStream_t)stream);
    if (rc) return rc;
    double* u_int = base;
    double* G = u_int + 3 * nc;
    double* T = G + 9 * nc;
    double* F = T + (c->law_mode != 0 ? 9 * nc : 0);
    double* Fn = F + 3 * (size_t)m.nflux;
    double* R_int = Fn + 3 * (size_t)m.ni;
    rc = jfnk::sync_load(c);
    if (!rc) rc = jfnk::perm_in(c, u, u_int);
    if (!rc) rc = jfnk::residual_bufs(c, u_int, R_int, jfnk::OUT_R, nullptr, G, T, F, Fn);
    if (!rc) rc = jfnk::perm_out(c, R_int, R);
    return rc;
}
