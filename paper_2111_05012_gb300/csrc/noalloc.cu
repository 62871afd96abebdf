// amg_apply_D_noalloc: the Wilson-clover stencil call of amg_apply_D with its
// two internal-layout work fields in a fixed static device array instead of
// library-allocated memory, for callers that cannot allocate device memory.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kernels.h"
#include "lqcd_amg.h"

// Work fields of amg_apply_D_noalloc: [input field | output field], each half
// of the array.  Held by every GPU that loads the library until exit.
#define AMG_NOALLOC_SCRATCH_BYTES (24u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[AMG_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// device address of the static array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, never a device address)
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

// Accessors for the handle fields needed here (defined in api.cu).
const GeomH* amg_internal_geom(const amg_dirac* d);
const void* amg_internal_links(const amg_dirac* d, int prec);
const void* amg_internal_clover(const amg_dirac* d, int prec);
double amg_internal_kappa(const amg_dirac* d);
void amg_internal_set_error(const char* msg);

extern "C" amg_status amg_apply_D_noalloc(amg_dirac* d, const void* in, void* out, int nrhs, amg_prec prec,
                                          amg_stream s) {
    if (!d || !in || !out || nrhs < 1) {
        amg_internal_set_error("amg_apply_D_noalloc: bad argument");
        return AMG_EINVAL;
    }
    if (prec != AMG_F64 && prec != AMG_F32 && prec != AMG_F16) {
        amg_internal_set_error("amg_apply_D_noalloc: prec must be AMG_F64, AMG_F32 or AMG_F16");
        return AMG_EINVAL;
    }
    const GeomH& g = *amg_internal_geom(d);
    const size_t field = fine_spinor_bytes((int)prec, g.V) * (size_t)nrhs;
    const size_t half = AMG_NOALLOC_SCRATCH_BYTES / 2;
    if (field > half) {
        std::string msg = "amg_apply_D_noalloc: " + std::to_string(field) + " bytes per work field exceed the " +
                          std::to_string(half) + "-byte limit (nrhs * volume too large for this entry point)";
        amg_internal_set_error(msg.c_str());
        return AMG_EINVAL;
    }
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        amg_internal_set_error((std::string("amg_apply_D_noalloc: cudaGetSymbolAddress -> ") + cudaGetErrorString(e)).c_str());
        return AMG_ECUDA;
    }
    void* win = base;
    void* wout = (unsigned char*)base + half;
    cudaStream_t st = (cudaStream_t)s;
    const int p = (int)prec;
    // both work fields are fully written before they are read: nothing to clear
    e = launch_pack_spinor(p, g, in, win, nrhs, st);
    if (e == cudaSuccess)
        e = launch_dirac(p, g, nullptr, amg_internal_links(d, p), amg_internal_clover(d, p), win, wout, nullptr,
                         amg_internal_kappa(d), nrhs, st);
    if (e == cudaSuccess) e = launch_unpack_spinor(p, g, wout, out, nrhs, st);
    if (e != cudaSuccess) {
        amg_internal_set_error((std::string("amg_apply_D_noalloc: ") + cudaGetErrorString(e)).c_str());
        return AMG_ECUDA;
    }
    return AMG_OK;
}
