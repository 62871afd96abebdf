// Gauge-equivariant parallel-transport convolution layers of the learned
// preconditioner:
//   out^a(x) = sum_b sum_d W_d^{ab} (T_d in^b)(x),
//   T_0 = 1, (T_{+mu} f)(x) = U_mu(x) f(x+mu), (T_{-mu} f)(x) = U_mu(x-mu)^dag f(x-mu)
// (fermion boundary phase on the t wrap), W_d^{ab} a complex 4x4 spin matrix
// stored in bfloat16 and applied with FP32 accumulation.  Fields are FP32
// internal spinors, C channels stored one after another.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kT = 256;
constexpr int kMaxC = 4;

Geom make_geom(const GeomH& h) {
    Geom g;
    for (int i = 0; i < 4; ++i) g.L[i] = h.L[i];
    g.stride[0] = 1;
    g.stride[1] = h.L[0];
    g.stride[2] = h.L[0] * h.L[1];
    g.stride[3] = h.L[0] * h.L[1] * h.L[2];
    g.V = h.V;
    g.antiperiodic = h.antiperiodic;
    return g;
}
int sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// (T_d f)(x) for a 12-component FP32 field f (channel base pointer)
DEV void transport(const Geom& g, const void* U, const void* f, int s, const int c[4], int d, cx<float> out[12]) {
    if (d == 0) {
        SpinorIO<P32>::load(f, g.V, s, out);
        return;
    }
    const int mu = (d - 1) & 3, dir = d <= 4 ? 1 : -1;
    float ph;
    const int n = neighbour(g, s, c, mu, dir, ph);
    cx<float> v[12], u[3][3];
    SpinorIO<P32>::load(f, g.V, n, v);
    GaugeIO<P32>::load(U, g.V, mu, dir > 0 ? s : n, u);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<float> t = czero<float>();
#pragma unroll
            for (int b = 0; b < 3; ++b) t = t + (dir > 0 ? u[a][b] * v[3 * sp + b] : cmulc(u[b][a], v[3 * sp + b]));
            out[3 * sp + a] = ph * t;
        }
}

// out^a = sum_b sum_d W[a][b][d] T_d in^b; weights bf16 [COUT][CIN][9][4][4][2]
template <int COUT>
__global__ void __launch_bounds__(kT) ptconv_forward_kernel(Geom g, int cin, const void* __restrict__ U,
                                                            const __nv_bfloat16* __restrict__ W, const void* in,
                                                            void* out) {
    __shared__ cx<float> w[kMaxC * kMaxC * 9 * 16];
    const int nw = COUT * cin * 9 * 16;
    for (int i = threadIdx.x; i < nw; i += blockDim.x)
        w[i] = {__bfloat162float(W[2 * i]), __bfloat162float(W[2 * i + 1])};
    __syncthreads();
    const size_t fb = spinor_bytes<P32>(g.V);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        int c[4];
        site_coords(g, s, c);
        cx<float> acc[COUT][12];
#pragma unroll
        for (int a = 0; a < COUT; ++a)
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[a][k] = czero<float>();
        for (int b = 0; b < cin; ++b) {
            const char* fin = (const char*)in + b * fb;
            for (int d = 0; d < 9; ++d) {
                cx<float> phi[12];
                transport(g, U, fin, s, c, d, phi);
#pragma unroll
                for (int a = 0; a < COUT; ++a) {
                    const cx<float>* wd = w + ((a * cin + b) * 9 + d) * 16;
#pragma unroll
                    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const cx<float> ws = wd[sp * 4 + t];
#pragma unroll
                            for (int col = 0; col < 3; ++col) cfma(acc[a][3 * sp + col], ws, phi[3 * t + col]);
                        }
                }
            }
        }
#pragma unroll
        for (int a = 0; a < COUT; ++a) SpinorIO<P32>::store((char*)out + a * fb, g.V, s, acc[a]);
    }
}

// Weight gradient G[a][b][d][s][t] = sum_{x,c} gout^a(x)[s,c] conj((T_d in^b)(x)[t,c]).
// blockIdx.y = b*9 + d; every CTA writes its partial sums (COUT*16 complex,
// accumulated in FP32 per thread, FP64 across the CTA) to part[y][blockIdx.x].
template <int COUT>
__global__ void __launch_bounds__(kT) ptconv_wgrad_kernel(Geom g, const void* __restrict__ U, const void* in,
                                                          const void* gout, double2* part) {
    __shared__ double red[COUT * 16 * 2][kT / 32];
    const int b = blockIdx.y / 9, d = blockIdx.y % 9;
    const size_t fb = spinor_bytes<P32>(g.V);
    cx<float> acc[COUT][16];
#pragma unroll
    for (int a = 0; a < COUT; ++a)
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[a][k] = czero<float>();
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        int c[4];
        site_coords(g, s, c);
        cx<float> phi[12];
        transport(g, U, (const char*)in + b * fb, s, c, d, phi);
#pragma unroll
        for (int a = 0; a < COUT; ++a) {
            cx<float> gv[12];
            SpinorIO<P32>::load((const char*)gout + a * fb, g.V, s, gv);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int t = 0; t < 4; ++t)
#pragma unroll
                    for (int col = 0; col < 3; ++col)
                        cfmac(acc[a][sp * 4 + t], phi[3 * t + col], gv[3 * sp + col]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < COUT; ++a)
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float re = warp_sum(acc[a][k].re), im = warp_sum(acc[a][k].im);
            if (lane == 0) {
                red[2 * (a * 16 + k)][warp] = re;
                red[2 * (a * 16 + k) + 1][warp] = im;
            }
        }
    __syncthreads();
    for (int q = threadIdx.x; q < COUT * 16; q += blockDim.x) {
        double re = 0, im = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            re += red[2 * q][w];
            im += red[2 * q + 1][w];
        }
        part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (COUT * 16) + q] = make_double2(re, im);
    }
}

// y = s * (y - e) and partial sums of |y - e|^2 (for the loss), flat float2 arrays
__global__ void residual_scale_kernel(float2* y, const float2* __restrict__ e, size_t n, float scale,
                                      double* part) {
    __shared__ double red[32];
    double acc = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float2 a = y[i], b = e[i];
        float dr = a.x - b.x, di = a.y - b.y;
        acc += (double)dr * dr + (double)di * di;
        y[i] = make_float2(scale * dr, scale * di);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

}  // namespace

int ptconv_grid() { return 2 * sms(); }

cudaError_t launch_ptconv_forward(const GeomH& gh, int cin, int cout, const void* U32, const void* Wbf16,
                                  const void* in, void* out, cudaStream_t st) {
    if (cin < 1 || cin > kMaxC || cout < 1 || cout > kMaxC) return cudaErrorInvalidValue;
    Geom g = make_geom(gh);
    int grid = (g.V + kT - 1) / kT;
    if (grid > sms() * 16) grid = sms() * 16;
    const __nv_bfloat16* W = (const __nv_bfloat16*)Wbf16;
    switch (cout) {
        case 1: (note_launch(), ptconv_forward_kernel<1><<<grid, kT, 0, st>>>(g, cin, U32, W, in, out)); break;
        case 2: (note_launch(), ptconv_forward_kernel<2><<<grid, kT, 0, st>>>(g, cin, U32, W, in, out)); break;
        case 3: (note_launch(), ptconv_forward_kernel<3><<<grid, kT, 0, st>>>(g, cin, U32, W, in, out)); break;
        default: (note_launch(), ptconv_forward_kernel<4><<<grid, kT, 0, st>>>(g, cin, U32, W, in, out)); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_ptconv_wgrad(const GeomH& gh, int cin, int cout, const void* U32, const void* in,
                                const void* gout, double2* part, cudaStream_t st) {
    if (cin < 1 || cin > kMaxC || cout < 1 || cout > kMaxC) return cudaErrorInvalidValue;
    Geom g = make_geom(gh);
    dim3 grid(ptconv_grid(), cin * 9);
    switch (cout) {
        case 1: (note_launch(), ptconv_wgrad_kernel<1><<<grid, kT, 0, st>>>(g, U32, in, gout, part)); break;
        case 2: (note_launch(), ptconv_wgrad_kernel<2><<<grid, kT, 0, st>>>(g, U32, in, gout, part)); break;
        case 3: (note_launch(), ptconv_wgrad_kernel<3><<<grid, kT, 0, st>>>(g, U32, in, gout, part)); break;
        default: (note_launch(), ptconv_wgrad_kernel<4><<<grid, kT, 0, st>>>(g, U32, in, gout, part)); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_residual_scale(void* y, const void* e, size_t n, float scale, double* part, cudaStream_t st) {
    (note_launch(), residual_scale_kernel<<<ptconv_grid(), kT, 0, st>>>((float2*)y, (const float2*)e, n, scale, part));
    return cudaGetLastError();
}
