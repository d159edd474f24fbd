// Allocation-free variant of the true-residual check (sgw_residual_noalloc).
//
// sgw_residual stages host buffers and grows the system's workspace with cudaMalloc.  Some
// callers cannot let a library allocate device memory on their behalf: a framework whose
// caching allocator or fixed arena owns every byte of device memory, or a code path that
// must not pay the device-wide synchronisation cudaFree can imply.  For them this entry
// point takes device buffers only and keeps its per-CTA scratch (two plane-wave vectors per
// CTA) in the file-scope array below, which every GPU that loads the library holds until
// the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <mutex>

#include "setup.h"
#include "sgw.h"
#include "sgw_internal.cuh"

namespace sgw {
sgw_status noalloc_fail(sgw_status s, const char* msg);
sgw_status noalloc_plan(const sgw_system* sys, const Plan** plan, int* dev);
}  // namespace sgw

using namespace sgw;

namespace {

// 4 MiB of scratch: 2 * n_pw complex values per vector owner (a CTA, or a cluster).
constexpr size_t kScratchElems = SGW_NOALLOC_SCRATCH_BYTES / sizeof(double2);
static __device__ __align__(256) double2 g_scratch[kScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double2* g_scratch_ptr[kMaxDevices] = {};   // device address of g_scratch on each device, once looked up

// Device memory of device `dev` (cudaMalloc, a memory pool of that device), or managed
// memory (reachable from every device).  Host memory, registered or not, and device memory of
// any other GPU are refused: the kernel would read another device's memory over the
// interconnect, or fault.
bool device_ptr(const void* p, int dev) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Makes `dev` current for the lifetime of the guard and then restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
        if (err != cudaSuccess) prev = -1;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" sgw_status sgw_residual_noalloc(sgw_system* sys, int nrhs, const void* rhs, const double* e_ref,
                                           int nomega, const double* omega, double eta, const void* dpsi,
                                           double* rel_res, double* cert, void* stream) {
    const Plan* P = nullptr;
    int dev = 0;
    sgw_status s = noalloc_plan(sys, &P, &dev);
    if (s != SGW_OK) return s;
    if (nrhs < 0 || nomega < 0) return noalloc_fail(SGW_EINVAL, "negative size");
    if (!(eta > 0.0)) return noalloc_fail(SGW_EINVAL, "eta must be positive");
    if (P->nocc == 0) return noalloc_fail(SGW_ESTATE, "sgw_set_occupied has not been called");
    const size_t np = (size_t)nrhs * nomega;
    if (np == 0) return SGW_OK;
    if (np > (size_t)INT_MAX) return noalloc_fail(SGW_EUNSUPPORTED, "nrhs * nomega above INT_MAX");
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(SGW_EUNSUPPORTED, "device index above 63");
    if (!device_ptr(rhs, dev) || !device_ptr(e_ref, dev) || !device_ptr(omega, dev) || !device_ptr(dpsi, dev) ||
        !device_ptr(rel_res, dev) || !device_ptr(cert, dev))
        return noalloc_fail(SGW_EINVAL,
                            "sgw_residual_noalloc takes device memory of the system's device (or managed memory) "
                            "only: it stages nothing");
    const size_t per_cta = 2 * (size_t)P->npw;
    if (per_cta > kScratchElems) {
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "n_pw = %d needs %zu bytes of scratch per CTA; the built-in scratch holds %zu bytes "
                      "(n_pw <= %zu)",
                      P->npw, per_cta * sizeof(double2), (size_t)SGW_NOALLOC_SCRATCH_BYTES, kScratchElems / 2);
        return noalloc_fail(SGW_EUNSUPPORTED, buf);
    }
    DeviceGuard guard(dev);   // the caller's current device is restored on return
    cudaError_t e = guard.err;
    if (e != cudaSuccess) return noalloc_fail(SGW_ECUDA, cudaGetErrorString(e));
    double2* scratch = nullptr;
    {
        // First call on this device: look up the device address of the scratch array (the
        // host-side name g_scratch is only a stand-in for it).
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) return noalloc_fail(SGW_ECUDA, cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<double2*>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    // owners: CTAs, or clusters of CTAs when the box is split over a cluster; each takes
    // 2 n_pw scratch values
    int owners = 0;
    e = residual_owners(*P, SGW_PREC_FP64, &owners);
    if (e != cudaSuccess) return noalloc_fail(SGW_ECUDA, cudaGetErrorString(e));
    owners = (int)std::min<size_t>({(size_t)owners, kScratchElems / per_cta, np});
    // The kernel writes every scratch element it reads before reading it: nothing to clear.
    e = launch_residual(*P, nrhs, nomega, nullptr, 0, (const double2*)rhs, e_ref, omega, eta, (const double2*)dpsi,
                        scratch, rel_res, cert, nullptr, owners, (cudaStream_t)stream);
    if (e != cudaSuccess) return noalloc_fail(SGW_ECUDA, cudaGetErrorString(e));
    return SGW_OK;
}
