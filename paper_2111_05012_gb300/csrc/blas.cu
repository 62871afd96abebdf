// BLAS-1 on flat complex arrays (double2 or float2) for the Krylov solvers.
// Reductions accumulate in FP64 and write one partial per CTA; the grid size
// is fixed (blas_grid()) so the final fixed-order sum is deterministic.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kMaxDots = 20;
constexpr int kBT = 256;

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int blas_grid_size() { return 2 * sm_count(); }

template <typename V> struct VT;
template <> struct VT<double2> { using T = double; };
template <> struct VT<float2> { using T = float; };

struct PtrList {
    const void* p[kMaxDots];
};
struct CoefList {
    double2 c[kMaxDots];
};

// K dots <a_j, b>, K a compile-time constant so that only K accumulation
// chains are issued (FP64 arithmetic is scarce on this part)
// K dots <a_j, b> (quantities 0..K-1) and, with NB, |b|^2 as quantity K (imaginary part 0)
// (the body of one CTA bx of gx; PL: anything with an indexable member p of vector pointers)
template <typename V, int K, bool NB, class PL>
DEV void multi_dot_body(const PL& a, const V* __restrict__ b, size_t n, double2* partials, int bx, int gx) {
    constexpr int NQ = K + (NB ? 1 : 0);
    __shared__ double red[2 * NQ * 32];
    double acc[2 * NQ];
#pragma unroll
    for (int j = 0; j < 2 * NQ; ++j) acc[j] = 0.0;
    for (size_t i = bx * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gx * blockDim.x) {
        V y = b[i];
        const double yr = y.x, yi = y.y;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            V x = ((const V*)a.p[j])[i];
            const double xr = x.x, xi = x.y;
            // conj(x) y as nested fused multiply-adds (two FP64 instructions per real accumulation)
            acc[2 * j] = fma(xr, yr, acc[2 * j]);
            acc[2 * j] = fma(xi, yi, acc[2 * j]);
            acc[2 * j + 1] = fma(xr, yi, acc[2 * j + 1]);
            acc[2 * j + 1] = fma(-xi, yr, acc[2 * j + 1]);
        }
        if (NB) {
            acc[2 * K] = fma(yr, yr, acc[2 * K]);
            acc[2 * K] = fma(yi, yi, acc[2 * K]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < 2 * NQ; ++j) {
        double v = warp_sum(acc[j]);
        if (lane == 0) red[j * 32 + warp] = v;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < NQ; j += blockDim.x) {
        double re = 0, im = 0;
        for (int w = 0; w < nw; ++w) {
            re += red[(2 * j) * 32 + w];
            im += red[(2 * j + 1) * 32 + w];
        }
        partials[(size_t)j * gx + bx] = make_double2(re, im);
    }
}
template <typename V, int K, bool NB>
__global__ void multi_dot_kernel(PtrList a, const V* __restrict__ b, size_t n, double2* partials) {
    multi_dot_body<V, K, NB>(a, b, n, partials, blockIdx.x, gridDim.x);
}

template <typename V, int K>
void multi_dot_launch(int k, bool nb, const PtrList& pl, const V* b, size_t n, double2* partials, cudaStream_t st) {
    if constexpr (K > 1) {
        if (k < K) return multi_dot_launch<V, K - 1>(k, nb, pl, b, n, partials, st);
    }
    if (nb) (note_launch(), multi_dot_kernel<V, K, true><<<blas_grid_size(), kBT, 0, st>>>(pl, b, n, partials));
    else (note_launch(), multi_dot_kernel<V, K, false><<<blas_grid_size(), kBT, 0, st>>>(pl, b, n, partials));
}

// y += sum_{j<K} c_j x_j, then partial dots <x_j, y_new> (DOT) or partial |y_new|^2:
// one pass over the vectors for the update of a Gram-Schmidt pass and the
// reduction of the next one
// the sum of the gridDim.x partials of each of k quantities ([j][gridDim.x]),
// one warp per quantity, lanes striding (fixed order: every CTA of the launch
// gets bitwise the same sums); out[j] = -sum (the update coefficient), and CTA
// 0 stores +sum in used[j] for the host's Hessenberg column
DEV void coefficients_from_partials(const double2* src, int k, double2* out, double2* used, int bx, int gx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < k; j += nw) {
        double re = 0, im = 0;
        for (int t = lane; t < gx; t += 32) {
            const double2 v = __ldcg(src + (size_t)j * gx + t);
            re += v.x;
            im += v.y;
        }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) {
            out[j] = make_double2(-re, -im);
            if (bx == 0 && used) used[j] = make_double2(re, im);
        }
    }
    __syncthreads();
}

template <typename V, int K, int MODE, class PL>   // MODE 0: |y|^2; 1: dots; 2: dots and |y|^2 (quantity K)
DEV void multi_axpy_reduce_body(const PL& x, V* y, size_t n, double2* partials, const double2* csrc, double2* cused,
                                int bx, int gx) {
    using T = typename VT<V>::T;
    constexpr bool DOT = MODE >= 1, NRM = MODE != 1;
    constexpr int NA = (DOT ? 2 * K : 0) + (NRM ? (DOT ? 2 : 1) : 0);
    __shared__ double red[NA * 32];
    __shared__ double2 cdev[K];
    // coefficients: minus the sums of the partials a previous reduction left at csrc
    // (summed here, so no host round trip)
    coefficients_from_partials(csrc, K, cdev, cused, bx, gx);
    T cre[K], cim[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        cre[j] = (T)cdev[j].x;
        cim[j] = (T)cdev[j].y;
    }
    double acc[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) acc[j] = 0.0;
    for (size_t i = bx * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gx * blockDim.x) {
        V xs[K];
#pragma unroll
        for (int j = 0; j < K; ++j) xs[j] = ((const V*)x.p[j])[i];
        V o = y[i];
        T re = o.x, im = o.y;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const T cr = cre[j], ci = cim[j];
            re = fma(cr, xs[j].x, re);
            re = fma(-ci, xs[j].y, re);
            im = fma(cr, xs[j].y, im);
            im = fma(ci, xs[j].x, im);
        }
        o.x = re;
        o.y = im;
        y[i] = o;
        if constexpr (DOT) {
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const double xr = xs[j].x, xi = xs[j].y;
                acc[2 * j] = fma(xr, (double)re, acc[2 * j]);
                acc[2 * j] = fma(xi, (double)im, acc[2 * j]);
                acc[2 * j + 1] = fma(xr, (double)im, acc[2 * j + 1]);
                acc[2 * j + 1] = fma(-xi, (double)re, acc[2 * j + 1]);
            }
        }
        if constexpr (NRM) {
            double& an = acc[DOT ? 2 * K : 0];
            an = fma((double)re, (double)re, an);
            an = fma((double)im, (double)im, an);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        double v = warp_sum(acc[j]);
        if (lane == 0) red[j * 32 + warp] = v;
    }
    __syncthreads();
    if (DOT) {
        constexpr int NQ = K + (NRM ? 1 : 0);   // the norm pair is (|y|^2, 0)
        for (int j = threadIdx.x; j < NQ; j += blockDim.x) {
            double re = 0, im = 0;
            for (int w = 0; w < nw; ++w) {
                re += red[(2 * j) * 32 + w];
                im += red[(2 * j + 1) * 32 + w];
            }
            partials[(size_t)j * gx + bx] = make_double2(re, im);
        }
    } else if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < nw; ++w) t += red[w];
        reinterpret_cast<double*>(partials)[bx] = t;
    }
}
template <typename V, int K, int MODE>
__global__ void multi_axpy_reduce_kernel(PtrList x, V* y, size_t n, double2* partials, const double2* csrc,
                                         double2* cused) {
    multi_axpy_reduce_body<V, K, MODE>(x, y, n, partials, csrc, cused, blockIdx.x, gridDim.x);
}

template <typename V, int K, int MODE>
void multi_axpy_reduce_launch(int k, const PtrList& pl, V* y, size_t n, double2* partials, const double2* csrc,
                              double2* cused, cudaStream_t st) {
    if constexpr (K > 1) {
        if (k < K) return multi_axpy_reduce_launch<V, K - 1, MODE>(k, pl, y, n, partials, csrc, cused, st);
    }
    (note_launch(), multi_axpy_reduce_kernel<V, K, MODE><<<blas_grid_size(), kBT, 0, st>>>(pl, y, n, partials, csrc,
                                                                                           cused));
}

template <typename V>
DEV void norm2_body(const V* __restrict__ a, size_t n, double* partials, int bx, int gx) {
    __shared__ double red[32];
    double acc = 0;
    for (size_t i = bx * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gx * blockDim.x) {
        V x = a[i];
        acc = fma((double)x.x, (double)x.x, acc);
        acc = fma((double)x.y, (double)x.y, acc);
    }
    acc = warp_sum(acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < nw; ++w) t += red[w];
        partials[bx] = t;
    }
}
template <typename V>
__global__ void norm2_kernel(const V* __restrict__ a, size_t n, double* partials) {
    norm2_body<V>(a, n, partials, blockIdx.x, gridDim.x);
}

template <typename V>
__global__ void axpby_kernel(double2 al, const V* __restrict__ x, double2 be, V* y, size_t n) {
    using T = typename VT<V>::T;
    const T ar = (T)al.x, ai = (T)al.y, br = (T)be.x, bi = (T)be.y;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        V a = x[i], b = y[i];
        V o;
        o.x = ar * a.x - ai * a.y + br * b.x - bi * b.y;
        o.y = ar * a.y + ai * a.x + br * b.y + bi * b.x;
        y[i] = o;
    }
}

// y = x / |x| with |x|^2 the sum of the gridDim.x partials in src (left by a
// norm reduction of the same grid); y = 0 if |x| = 0.  CTA 0 stores |x| in hn.
// Two multiplications per complex entry.
template <typename V>
DEV void normalise_body(const double* src, double* hn, const V* __restrict__ x, V* y, size_t n, int bx, int gx) {
    using T = typename VT<V>::T;
    __shared__ double s_inv;
    if (threadIdx.x < 32) {
        double t = 0;
        for (int k = threadIdx.x; k < gx; k += 32) t += __ldcg(src + k);
        t = warp_sum(t);
        if (threadIdx.x == 0) {
            const double h = sqrt(t);
            s_inv = h > 0 ? 1.0 / h : 0.0;
            if (bx == 0) *hn = h;
        }
    }
    __syncthreads();
    const T a = (T)s_inv;
    for (size_t i = bx * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gx * blockDim.x) {
        V v = x[i];
        v.x *= a;
        v.y *= a;
        y[i] = v;
    }
}
template <typename V>
__global__ void normalise_kernel(const double* src, double* hn, const V* __restrict__ x, V* y, size_t n) {
    normalise_body<V>(src, hn, x, y, n, blockIdx.x, gridDim.x);
}

// y = a x for a real a (two multiplications per complex entry)
template <typename V>
__global__ void scale_real_kernel(double a, const V* __restrict__ x, V* y, size_t n) {
    using T = typename VT<V>::T;
    const T ar = (T)a;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        V v = x[i];
        v.x *= ar;
        v.y *= ar;
        y[i] = v;
    }
}

template <typename V>
__global__ void multi_axpy_kernel(int k, CoefList c, PtrList x, V* y, size_t n) {
    using T = typename VT<V>::T;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        V o = y[i];
        T re = o.x, im = o.y;
        for (int j = 0; j < k; ++j) {
            V a = ((const V*)x.p[j])[i];
            T cr = (T)c.c[j].x, ci = (T)c.c[j].y;
            re = fma(cr, a.x, re);
            re = fma(-ci, a.y, re);
            im = fma(cr, a.y, im);
            im = fma(ci, a.x, im);
        }
        o.x = re;
        o.y = im;
        y[i] = o;
    }
}

// ---- ragged batch: one Gram-Schmidt pass for every problem, one launch per step
// (per problem: basis V_0..V_j, w, its own partials and coefficients; CTA ranges
// from the prefix table, the same ranges in all three launches of a pass)
struct BasisView {
    const void* const* p;
};
template <int K>
__global__ void __launch_bounds__(kBT) gs_dot_ragged_kernel(const RaggedDev* __restrict__ d,
                                                            const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    multi_dot_body<double2, K, false>(BasisView{q.basis}, (const double2*)q.w, q.n, q.gs_part, bx, gx);
}
template <int K>
__global__ void __launch_bounds__(kBT) gs_update_ragged_kernel(const RaggedDev* __restrict__ d,
                                                               const int* __restrict__ off, int np, int pass) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    multi_axpy_reduce_body<double2, K, 0>(BasisView{q.basis}, (double2*)q.w, q.n, q.gs_part + 2 * q.R, q.gs_part,
                                          q.gs_coef + 32 * pass, bx, gx);
}
__global__ void __launch_bounds__(kBT) gs_normalise_ragged_kernel(const RaggedDev* __restrict__ d,
                                                                  const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    normalise_body<double2>((const double*)(q.gs_part + 2 * q.R), (double*)(q.gs_coef + 63), (const double2*)q.w,
                            (double2*)q.vnext, q.n, bx, gx);
}
// restart: |rsrc|^2 partials, then basis[0] = rsrc / |rsrc| and nval = |rsrc|
__global__ void __launch_bounds__(kBT) rnorm_ragged_kernel(const RaggedDev* __restrict__ d,
                                                           const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    norm2_body<double2>((const double2*)q.rsrc, q.n, q.npart, bx, gx);
}
__global__ void __launch_bounds__(kBT) rnormalise_ragged_kernel(const RaggedDev* __restrict__ d,
                                                                const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    normalise_body<double2>(q.npart, q.nval, (const double2*)q.rsrc, (double2*)const_cast<void*>(q.basis[0]), q.n,
                            bx, gx);
}
template <int K>
void gs_ragged_launch(int k, int step, const RaggedDev* d, const int* off, int np, int ctas, int pass,
                      cudaStream_t st) {
    if constexpr (K > 1) {
        if (k < K) return gs_ragged_launch<K - 1>(k, step, d, off, np, ctas, pass, st);
    }
    if (step == 0) (note_launch(), gs_dot_ragged_kernel<K><<<ctas, kBT, 0, st>>>(d, off, np));
    else (note_launch(), gs_update_ragged_kernel<K><<<ctas, kBT, 0, st>>>(d, off, np, pass));
}

}  // namespace

int blas_grid() { return blas_grid_size(); }

cudaError_t launch_multi_dot(int prec, int k, const void* const* a, const void* b, size_t n, double2* partials,
                             cudaStream_t st) {
    if (k > kMaxDots) return cudaErrorInvalidValue;
    PtrList pl;
    for (int j = 0; j < k; ++j) pl.p[j] = a[j];
    if (k < 1) return cudaErrorInvalidValue;
    if (prec == 0) multi_dot_launch<double2, kMaxDots>(k, false, pl, (const double2*)b, n, partials, st);
    else multi_dot_launch<float2, kMaxDots>(k, false, pl, (const float2*)b, n, partials, st);
    return cudaGetLastError();
}
cudaError_t launch_multi_dot_norm(int prec, int k, const void* const* a, const void* b, size_t n, double2* partials,
                                  cudaStream_t st) {
    if (k < 1 || k >= kMaxDots) return cudaErrorInvalidValue;
    PtrList pl;
    for (int j = 0; j < k; ++j) pl.p[j] = a[j];
    if (prec == 0) multi_dot_launch<double2, kMaxDots - 1>(k, true, pl, (const double2*)b, n, partials, st);
    else multi_dot_launch<float2, kMaxDots - 1>(k, true, pl, (const float2*)b, n, partials, st);
    return cudaGetLastError();
}
cudaError_t launch_norm2(int prec, const void* a, size_t n, double* partials, cudaStream_t st) {
    if (prec == 0) (note_launch(), norm2_kernel<double2><<<blas_grid(), kBT, 0, st>>>((const double2*)a, n, partials));
    else (note_launch(), norm2_kernel<float2><<<blas_grid(), kBT, 0, st>>>((const float2*)a, n, partials));
    return cudaGetLastError();
}
cudaError_t launch_axpby(int prec, double2 al, const void* x, double2 be, void* y, size_t n, cudaStream_t st) {
    if (prec == 0) (note_launch(), axpby_kernel<double2><<<blas_grid(), kBT, 0, st>>>(al, (const double2*)x, be, (double2*)y, n));
    else (note_launch(), axpby_kernel<float2><<<blas_grid(), kBT, 0, st>>>(al, (const float2*)x, be, (float2*)y, n));
    return cudaGetLastError();
}
cudaError_t launch_multi_axpy(int prec, int k, const double2* c, const void* const* x, void* y, size_t n,
                              cudaStream_t st) {
    if (k > kMaxDots) return cudaErrorInvalidValue;
    CoefList cl;
    PtrList pl;
    for (int j = 0; j < k; ++j) {
        cl.c[j] = c[j];
        pl.p[j] = x[j];
    }
    if (prec == 0) (note_launch(), multi_axpy_kernel<double2><<<blas_grid(), kBT, 0, st>>>(k, cl, pl, (double2*)y, n));
    else (note_launch(), multi_axpy_kernel<float2><<<blas_grid(), kBT, 0, st>>>(k, cl, pl, (float2*)y, n));
    return cudaGetLastError();
}

cudaError_t launch_normalise(int prec, const double* norm_partials, double* hn, const void* x, void* y, size_t n,
                             cudaStream_t st) {
    if (prec == 0)
        (note_launch(), normalise_kernel<double2><<<blas_grid(), kBT, 0, st>>>(norm_partials, hn, (const double2*)x,
                                                                            (double2*)y, n));
    else
        (note_launch(), normalise_kernel<float2><<<blas_grid(), kBT, 0, st>>>(norm_partials, hn, (const float2*)x,
                                                                           (float2*)y, n));
    return cudaGetLastError();
}
cudaError_t launch_scale_real(int prec, double a, const void* x, void* y, size_t n, cudaStream_t st) {
    if (prec == 0)
        (note_launch(), scale_real_kernel<double2><<<blas_grid(), kBT, 0, st>>>(a, (const double2*)x, (double2*)y, n));
    else (note_launch(), scale_real_kernel<float2><<<blas_grid(), kBT, 0, st>>>(a, (const float2*)x, (float2*)y, n));
    return cudaGetLastError();
}

cudaError_t launch_multi_axpy_reduce_dev(int prec, int k, const double2* csrc, double2* cused, const void* const* x,
                                         void* y, size_t n, int mode, double2* partials, cudaStream_t st) {
    if (k < 1 || k > kMaxDots || (mode == 2 && k >= kMaxDots) || !csrc) return cudaErrorInvalidValue;
    PtrList pl;
    for (int j = 0; j < k; ++j) pl.p[j] = x[j];
#define MAR(V, M) \
    multi_axpy_reduce_launch<V, (M == 2 ? kMaxDots - 1 : kMaxDots), M>(k, pl, (V*)y, n, partials, csrc, cused, st)
    if (prec == 0) {
        if (mode == 0) MAR(double2, 0);
        else if (mode == 1) MAR(double2, 1);
        else MAR(double2, 2);
    } else {
        if (mode == 0) MAR(float2, 0);
        else if (mode == 1) MAR(float2, 1);
        else MAR(float2, 2);
    }
#undef MAR
    return cudaGetLastError();
}

// one classical Gram-Schmidt pass of step j (k = j + 1 basis vectors) for every problem of a
// ragged batch: partial dots <V_i, w>; w -= sum_i h_i V_i with |w'|^2 partials (h_i stored in
// gs_coef[32 pass + i]); V_{j+1} = w' / |w'| (|w'| in gs_coef[63])
cudaError_t launch_gs_ragged(int k, const void* d, const int* off, int np, int ctas, int pass, cudaStream_t st) {
    if (k < 1 || k > kMaxDots || ctas < 1) return cudaErrorInvalidValue;
    const RaggedDev* dd = (const RaggedDev*)d;
    gs_ragged_launch<kMaxDots>(k, 0, dd, off, np, ctas, pass, st);
    gs_ragged_launch<kMaxDots>(k, 1, dd, off, np, ctas, pass, st);
    (note_launch(), gs_normalise_ragged_kernel<<<ctas, kBT, 0, st>>>(dd, off, np));
    return cudaGetLastError();
}
int ragged_blas_ctas(size_t n) {
    const size_t per = (size_t)kBT * 16;   // about 16 entries per thread
    size_t c = (n + per - 1) / per;
    const size_t cap = (size_t)blas_grid_size();
    return (int)(c < 1 ? 1 : (c > cap ? cap : c));
}
cudaError_t launch_norm_v0_ragged(const void* d, const int* off, int np, int ctas, cudaStream_t st) {
    const RaggedDev* dd = (const RaggedDev*)d;
    (note_launch(), rnorm_ragged_kernel<<<ctas, kBT, 0, st>>>(dd, off, np));
    (note_launch(), rnormalise_ragged_kernel<<<ctas, kBT, 0, st>>>(dd, off, np));
    return cudaGetLastError();
}
