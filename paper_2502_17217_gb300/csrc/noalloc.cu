// jfnk_residual_noalloc: the residual R(u) evaluated without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a residual: code that
// runs while a CUDA stream is being captured into a graph (cudaMalloc is not allowed during
// capture), code in processes where another framework's pool owns the device memory, and
// latency-sensitive loops that must not take the implicit device synchronisation of
// cudaMalloc/cudaFree.  For them this entry point takes its scratch (the load factor, the
// caller-order to internal-order copies of u and R, the cell gradients, the large-strain
// traction operators and the two face-flux arrays) from one file-scope device array of fixed
// size instead of the context's buffers.  The caller still passes u and R.
//
// Properties a caller must know:
//  * the array holds kNoallocScratchDoubles doubles (16 MiB) and stays resident on every GPU
//    that loads the library, until the process exits;
//  * all calls share it and it keeps the contents of the last call; every element a call
//    reads it first writes, so nothing needs clearing between calls;
//  * calls whose work overlaps on the GPU (different streams, or several contexts on one
//    device) race on the array: serialise them;
//  * the first call on a device looks up the array's device address (cudaGetSymbolAddress)
//    with that device current; make that first call before any stream capture;
//  * the load factor is handed to the GPU as a kernel argument written into the array, so
//    the call never waits on the host and never touches the context's own copy of it; work
//    recorded from a call (for instance a captured graph) keeps the load factor of that call.
#include <mutex>

#include "device_common.cuh"
#include "jfnk_internal.h"

namespace {

constexpr size_t kNoallocScratchDoubles = size_t(1) << 21;  // 16 MiB
constexpr size_t kHeadDoubles = 32;                          // load factor slot, 256-byte padded
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

__global__ void k_noalloc_set_load(double* slot, double load)
{
    JF_PDL_ENTRY();  // the previous call's kernels have finished reading the slot
    *slot = load;
}

// true when p is memory the context's device can address from a kernel: device memory of
// that device, or managed memory
bool device_reachable(const void* p, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the (non-sticky) error the query left behind
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace

extern "C" int jfnk_residual_noalloc(jfnk_ctx* c, const double* u, double* R, void* stream)
{
    if (!c) return JFNK_EINVAL;
    if (!u || !R) return jfnk_fail(c, JFNK_EINVAL, "jfnk_residual_noalloc: u and R must not be NULL");
    if (c->dirty || !c->gdev)
        return jfnk_fail(c, JFNK_ESTATE, "jfnk_residual_noalloc: call jfnk_setup() first (this entry point never allocates)");
    const jfnk::DevMesh& m = c->dm;
    const size_t nc = (size_t)m.nc;
    const size_t need = kHeadDoubles + 3 * nc + 9 * nc + (c->law_mode != 0 ? 9 * nc : 0) + 3 * (size_t)m.nflux +
                        3 * (size_t)m.ni + 3 * nc;
    if (need > kNoallocScratchDoubles)
        return jfnk_fail(c, JFNK_EINVAL,
                         "jfnk_residual_noalloc: the mesh needs " + std::to_string(need) + " scratch doubles, more than the " +
                             std::to_string(kNoallocScratchDoubles) + " of the fixed array (use jfnk_residual)");
    if (cudaSetDevice(c->opt.device) != cudaSuccess) return jfnk_cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    if (!device_reachable(u, c->opt.device) || !device_reachable(R, c->opt.device))
        return jfnk_fail(c, JFNK_EINVAL,
                         "jfnk_residual_noalloc: u and R must be device (or managed) memory of the context's device");
    cudaError_t e;
    double* base = scratch_address(c->opt.device, &e);
    if (!base) return jfnk_cuda_fail(c, e, "cudaGetSymbolAddress");
    int rc = jfnk_use_stream(c, (cudaStream_t)stream);
    if (rc) return rc;
    double* load = base;
    double* u_int = base + kHeadDoubles;
    double* G = u_int + 3 * nc;
    double* T = G + 9 * nc;
    double* F = T + (c->law_mode != 0 ? 9 * nc : 0);
    double* Fn = F + 3 * (size_t)m.nflux;
    double* R_int = Fn + 3 * (size_t)m.ni;
    jfnk_launch(c, k_noalloc_set_load, dim3(1), dim3(1), load, c->load);
    JF_LAUNCHED(c);
    rc = jfnk::perm_in(c, u, u_int);
    if (!rc) rc = jfnk::residual_bufs(c, u_int, R_int, jfnk::OUT_R, nullptr, G, T, F, Fn, load);
    if (!rc) rc = jfnk::perm_out(c, R_int, R);
    return rc;
}
