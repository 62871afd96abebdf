// Seeded synthetic inputs generated on the device.
//
// The paper measures on gauge ensembles that are not available here; every
// workload of this library is a synthetic field U_mu(x) = exp(i eps H) with H
// a traceless Hermitian matrix of Gaussian entries, and Gaussian test vectors
// and right-hand sides.  The random numbers come from one counter-based
// generator, so any element can be drawn independently and the same element
// has the same value wherever it is drawn:
//
//   SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
//   generators", OOPSLA 2014) in counter mode: the n-th 64-bit word of the
//   stream with key k is mix64(k + (n + 1) * 0x9E3779B97F4A7C15), with the
//   published SplitMix64 finaliser mix64; the key of (seed, stream) is
//   mix64(seed * 0x9E3779B97F4A7C15 + stream).  A word w becomes the double
//   ((w >> 11) + 1) * 2^-53 in (0, 1].  Complex normal m of a stream is the
//   Box-Muller pair of words 2m, 2m+1: sqrt(-2 ln u0) (cos, sin)(2 pi u1).
//
// Link (site s, direction mu) takes complex normals 9 (4 s + mu) .. + 8 of
// the gauge stream as the row-major entries of A; H = (A + A^dag)/2 minus
// its trace/3.  exp(i eps H) is evaluated from the eigenvalues of Q = eps H
// (trigonometric solution of the characteristic cubic of a 3x3 Hermitian
// matrix) by Newton's divided-difference form of the interpolating
// polynomial, exp(iQ) = f[a] + f[a,b](Q - a) + f[a,b,c](Q - a)(Q - b) with
// f(x) = exp(ix) and a >= b >= c the eigenvalues: exact for any three nodes
// equal to the spectrum, and free of cancellation because
// f[a,b] = i exp(i(a+b)/2) sin(d)/d with d = (a-b)/2, and the error of
// f[a,b,c] is multiplied by (Q - a)(Q - b), which is small exactly when
// a - c is.  The result is unitary with unit determinant to rounding.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr int kThreads = 256;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

__device__ __forceinline__ double unit_open(uint64_t w) { return ((double)(w >> 11) + 1.0) * 0x1.0p-53; }

// complex normal m of the stream with key `key` (re, im)
__device__ __forceinline__ double2 complex_normal(uint64_t key, uint64_t m) {
    const double u0 = unit_open(mix64(key + (2 * m + 1) * kGolden));
    const double u1 = unit_open(mix64(key + (2 * m + 2) * kGolden));
    const double rad = sqrt(-2.0 * log(u0));
    const double ang = (2.0 * 3.141592653589793) * u1;
    double sn, cs;
    sincos(ang, &sn, &cs);
    return make_double2(rad * cs, rad * sn);
}

struct C {
    double re, im;
};
__device__ __forceinline__ C cadd(C a, C b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ C cmul(C a, C b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ C cscale(C a, double s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ C cexpi(double x) {
    double s, c;
    sincos(x, &s, &c);
    return {c, s};
}

// sin(d)/d, with its Taylor polynomial near 0 (error below 1e-17 there)
__device__ __forceinline__ double sinc(double d) {
    if (fabs(d) < 1e-4) {
        const double d2 = d * d;
        return 1.0 - d2 / 6.0 + d2 * d2 / 120.0;
    }
    return sin(d) / d;
}

// U = exp(i Q) for Hermitian Q (3x3, row-major)
__device__ void expi_hermitian3(const C Q[9], C U[9]) {
    // eigenvalues: Q = m + B, B traceless; lambda = m + 2p cos(phi + 2 pi k / 3), cos(3 phi) = det B / (2 p^3)
    const double m = (Q[0].re + Q[4].re + Q[8].re) / 3.0;
    C B[9];
    for (int k = 0; k < 9; ++k) B[k] = Q[k];
    B[0].re -= m;
    B[4].re -= m;
    B[8].re -= m;
    double tr2 = 0;   // tr(B^2) = sum |B_ij|^2 for Hermitian B
    for (int k = 0; k < 9; ++k) tr2 += B[k].re * B[k].re + B[k].im * B[k].im;
    const double p = sqrt(tr2 / 6.0);
    double a = m, b = m, c = m;
    if (p > 0) {
        // det B (real for Hermitian B)
        const C m0 = cadd(cmul(B[4], B[8]), cscale(cmul(B[5], B[7]), -1.0));
        const C m1 = cadd(cmul(B[3], B[8]), cscale(cmul(B[5], B[6]), -1.0));
        const C m2 = cadd(cmul(B[3], B[7]), cscale(cmul(B[4], B[6]), -1.0));
        const double det = cmul(B[0], m0).re - cmul(B[1], m1).re + cmul(B[2], m2).re;
        double r = det / (2.0 * p * p * p);
        r = fmin(1.0, fmax(-1.0, r));
        const double phi = acos(r) / 3.0;
        a = m + 2.0 * p * cos(phi);
        c = m + 2.0 * p * cos(phi + 2.0 * 3.141592653589793 / 3.0);
        b = 3.0 * m - a - c;
    }
    const C fa = cexpi(a);
    const C fab = cmul({0.0, 1.0}, cscale(cexpi(0.5 * (a + b)), sinc(0.5 * (a - b))));
    const C fbc = cmul({0.0, 1.0}, cscale(cexpi(0.5 * (b + c)), sinc(0.5 * (b - c))));
    const double den = a - c;
    C fabc;
    if (den < 1e-12 * (1.0 + fabs(a))) fabc = cscale(fa, -0.5);   // f''(a)/2: all three nodes coincide
    else fabc = cscale(cadd(fab, cscale(fbc, -1.0)), 1.0 / den);
    // QA = Q - a, QB = Q - b, U = fa + fab QA + fabc QA QB
    C QA[9], QB[9];
    for (int k = 0; k < 9; ++k) QA[k] = QB[k] = Q[k];
    for (int i = 0; i < 3; ++i) {
        QA[4 * i].re -= a;
        QB[4 * i].re -= b;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            C s = {0, 0};
            for (int k = 0; k < 3; ++k) s = cadd(s, cmul(QA[3 * i + k], QB[3 * k + j]));
            C u = cadd(cmul(fab, QA[3 * i + j]), cmul(fabc, s));
            if (i == j) u = cadd(u, fa);
            U[3 * i + j] = u;
        }
}

__global__ void random_normal_kernel(uint64_t key, uint64_t start, uint64_t count, double2* out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = complex_normal(key, start + i);
}

// one thread per link; canonical [site][mu][3][3][re, im] doubles
__global__ void gauge_random_kernel(uint64_t nlinks, double eps, uint64_t key, double2* canon) {
    for (uint64_t l = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; l < nlinks;
         l += (uint64_t)gridDim.x * blockDim.x) {
        C A[9];
        for (int e = 0; e < 9; ++e) {
            const double2 z = complex_normal(key, 9 * l + e);
            A[e] = {z.x, z.y};
        }
        C H[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                H[3 * i + j] = {0.5 * (A[3 * i + j].re + A[3 * j + i].re), 0.5 * (A[3 * i + j].im - A[3 * j + i].im)};
        const double tr = (H[0].re + H[4].re + H[8].re) / 3.0;
        for (int i = 0; i < 3; ++i) H[4 * i].re -= tr;
        for (int k = 0; k < 9; ++k) H[k] = cscale(H[k], eps);
        C U[9];
        expi_hermitian3(H, U);
        for (int e = 0; e < 9; ++e) canon[9 * l + e] = make_double2(U[e].re, U[e].im);
    }
}

// internal FP64 links [mu][9][site] (double2) -> canonical [site][mu][9]
__global__ void gauge_unpack64_kernel(int V, const double2* __restrict__ in, double2* out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    for (int mu = 0; mu < 4; ++mu)
        for (int e = 0; e < 9; ++e) out[((size_t)s * 4 + mu) * 9 + e] = in[((size_t)mu * 9 + e) * V + s];
}

int grid_for_count(uint64_t n) {
    uint64_t b = (n + kThreads - 1) / kThreads;
    const uint64_t cap = 152ull * 64;   // grid-stride loops beyond this
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

uint64_t rng_stream_key(uint64_t seed, uint64_t stream) { return mix64(seed * kGolden + stream); }

cudaError_t launch_random_normal(uint64_t seed, uint64_t stream, uint64_t start, uint64_t count, double* out,
                                 cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    (note_launch(), random_normal_kernel<<<grid_for_count(count), kThreads, 0, s>>>(
                        rng_stream_key(seed, stream), start, count, reinterpret_cast<double2*>(out)));
    return cudaGetLastError();
}

cudaError_t launch_gauge_random(const GeomH& g, double eps, uint64_t seed, uint64_t stream, double* canon,
                                cudaStream_t s) {
    const uint64_t nlinks = 4ull * (uint64_t)g.V;
    (note_launch(), gauge_random_kernel<<<grid_for_count(nlinks), kThreads, 0, s>>>(
                        nlinks, eps, rng_stream_key(seed, stream), reinterpret_cast<double2*>(canon)));
    return cudaGetLastError();
}

cudaError_t launch_gauge_unpack64(const GeomH& g, const void* U64, double* canon, cudaStream_t s) {
    (note_launch(), gauge_unpack64_kernel<<<(g.V + kThreads - 1) / kThreads, kThreads, 0, s>>>(
                        g.V, reinterpret_cast<const double2*>(U64), reinterpret_cast<double2*>(canon)));
    return cudaGetLastError();
}
