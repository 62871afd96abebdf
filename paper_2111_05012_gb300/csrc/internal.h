// Host-side internals shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "kernels.h"
#include "lqcd_amg.h"

// Owning device buffer that only grows.
struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) {
        o.p = nullptr;
        o.n = 0;
    }
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t ensure(size_t bytes) {
        if (bytes <= n) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
        if (e == cudaSuccess) n = bytes;
        return e;
    }
    template <typename T> T* as() const { return (T*)p; }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void swap(DevBuf& o) noexcept {
        void* tp = p;
        p = o.p;
        o.p = tp;
        size_t tn = n;
        n = o.n;
        o.n = tn;
    }
};

#define AMG_NN_MAX_LAYERS 4

// Learned parallel-transport preconditioner (layers of ptconv.cu).
struct amg_nn {
    amg_dirac* d = nullptr;
    int nlayers = 0;
    int ch[AMG_NN_MAX_LAYERS + 1] = {0};
    std::vector<std::vector<float>> w;      // FP32 master weights [cout][cin][9][4][4][re,im]
    std::vector<std::vector<double>> m, v;  // Adam moments
    int adam_t = 0;
    DevBuf wbf[AMG_NN_MAX_LAYERS];          // bfloat16 weights of the forward layers
    DevBuf wadj[AMG_NN_MAX_LAYERS];         // bfloat16 adjoint weights (input gradient)
    DevBuf act[AMG_NN_MAX_LAYERS + 1];      // activations, FP32 internal fields x channels
    DevBuf gbuf[2];                         // gradient fields
    DevBuf ework;                           // target field
    DevBuf part;                            // reduction partials
    DevBuf canon;                           // canonical staging
    double* hpart = nullptr;                // pinned partials
    ~amg_nn() {
        if (hpart) cudaFreeHost(hpart);
    }
};

// accessors implemented in api.cu
const GeomH* amg_internal_geom(const amg_dirac* d);
amg_dirac* amg_internal_hierarchy_dirac(amg_hierarchy* h);
const void* amg_internal_links(const amg_dirac* d, int prec);
void amg_internal_set_error(const char* msg);

// PT-conv launchers (ptconv.cu)
int ptconv_grid();
cudaError_t launch_ptconv_forward(const GeomH& g, int cin, int cout, const void* U32, const void* Wbf16,
                                  const void* in, void* out, cudaStream_t s);
cudaError_t launch_ptconv_wgrad(const GeomH& g, int cin, int cout, const void* U32, const void* in, const void* gout,
                                double2* part, cudaStream_t s);
cudaError_t launch_residual_scale(void* y, const void* e, size_t n, float scale, double* part, cudaStream_t s);

// network forward on FP32 internal fields: out = N(in) (nn_api.cu)
amg_status nn_forward_internal(amg_nn* nn, const void* in32, void* out32, cudaStream_t s);
