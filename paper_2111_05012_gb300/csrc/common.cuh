// Device-side building blocks shared by the kernels of the library:
// complex arithmetic, precision tags with their storage formats, lattice
// geometry and the spin-projected Wilson hop of Eq. 1.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#define HD __host__ __device__ __forceinline__
#define DEV __device__ __forceinline__

// ---------------------------------------------------------------- complex
template <typename T>
struct cx {
    T re, im;
};
template <typename T> HD cx<T> mkc(T r, T i) { return cx<T>{r, i}; }
template <typename T> HD cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> HD cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> HD cx<T> operator-(cx<T> a) { return {-a.re, -a.im}; }
template <typename T> HD cx<T> operator*(cx<T> a, cx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> HD cx<T> operator*(T s, cx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> HD cx<T> conj(cx<T> a) { return {a.re, -a.im}; }
// conj(a) * b
template <typename T> HD cx<T> cmulc(cx<T> a, cx<T> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// i * a
template <typename T> HD cx<T> timesI(cx<T> a) { return {-a.im, a.re}; }
template <typename T> HD T norm2(cx<T> a) { return a.re * a.re + a.im * a.im; }
template <typename T> HD cx<T> czero() { return {T(0), T(0)}; }
// acc += a b, acc += conj(a) b and acc += s a (s real) as fused multiply-adds:
// written as acc + a * b the product is formed first and then added, two
// extra instructions per complex multiply-accumulate
template <typename T> HD void cfma(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
template <typename T> HD void cfmac(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}
template <typename T> HD void rfma(cx<T>& acc, T s, cx<T> a) {
    acc.re = fma(s, a.re, acc.re);
    acc.im = fma(s, a.im, acc.im);
}
template <typename T, typename U> HD cx<T> ccast(cx<U> a) { return {T(a.re), T(a.im)}; }

// ---------------------------------------------------------------- double-float
// An unevaluated sum hi + lo of two floats (about 48 significant bits),
// with Knuth's two-sum and the FMA-based exact product (Dekker's
// splitting is not needed with a fused multiply-add).  Used where an FP64
// accurate result is needed but the FP64 pipe (1/64 of FP32 on this part)
// would be the bottleneck.
struct dfloat {
    float hi, lo;
    HD dfloat() : hi(0.f), lo(0.f) {}
    HD dfloat(float h) : hi(h), lo(0.f) {}
    HD dfloat(float h, float l) : hi(h), lo(l) {}
};
DEV dfloat two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
DEV dfloat quick_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
DEV dfloat operator+(dfloat x, dfloat y) {
    dfloat s = two_sum(x.hi, y.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return quick_two_sum(s.hi, e);
}
DEV dfloat operator-(dfloat x) { return {-x.hi, -x.lo}; }
DEV dfloat operator-(dfloat x, dfloat y) { return x + (-y); }
DEV dfloat operator*(dfloat x, dfloat y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
    return quick_two_sum(p, e);
}
DEV dfloat& operator+=(dfloat& x, dfloat y) { return x = x + y; }
DEV double to_double(dfloat x) { return (double)x.hi + (double)x.lo; }
HD dfloat split_double(double v) {
    float h = (float)v;
    return {h, (float)(v - (double)h)};
}
// FP64 <-> float pairs without FP64 instructions (double-precision conversions and
// subtractions run on the scarce FP64 pipe here).  split_double_bits: hi = the leading 24
// significant bits of v (truncated, exact), lo = the next 23 bits, |v - (hi + lo)| <
// 2^-46 |v|.  Values below 2^-126 in magnitude are dropped, lo below 2^-81 |v| scale likewise
// (absolute errors under 1e-31 against vectors of order one); infinities and NaNs stay
// infinite or NaN in hi.
DEV dfloat split_double_bits(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hw = (unsigned)(b >> 32), sign = hw & 0x80000000u;
    const int e = (int)((hw >> 20) & 0x7FF);   // biased exponent
    if (e < 1023 - 126) return dfloat(0.f, 0.f);
    if (e >= 1023 + 128) return dfloat(__uint_as_float(sign | 0x7F800000u | ((e == 2047 && (b << 12)) ? 0x400000u : 0u)), 0.f);
    const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
    float lo = 0.f;
    const int le = e - 1075 + 6 + 127;   // float exponent of 2^(e - 1075 + 6)
    if (le > 0) {
        // the 23 bits below hi as an exact float in [0, 2^23), scaled into place
        const float m = __fsub_rn(__uint_as_float(0x4B000000u | (unsigned)((b & 0x1FFFFFFFull) >> 6)), 8388608.f);
        lo = __fmul_rn(m, __uint_as_float((unsigned)le << 23));
        if (sign) lo = -lo;
    }
    return dfloat(hi, lo);
}
// the double of a float (exact; zero and subnormal floats give zero), integer instructions only
DEV double float_to_double_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    if (e == 0) return __longlong_as_double((long long)sign);
    const unsigned long long ed = e == 255 ? 2047ull : (unsigned long long)(e + 896);
    return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
// hi + lo rounded to a double: one FP64 addition
DEV double pair_to_double(float hi, float lo) { return float_to_double_bits(hi) + float_to_double_bits(lo); }


// ---------------------------------------------------------------- precision tags
// A tag fixes the storage of fine fields (spinor, links, clover) and the
// arithmetic type T.
struct P64 { using T = double; static constexpr int id = 0; };
struct P32 { using T = float; static constexpr int id = 1; };
struct P16 { using T = float; static constexpr int id = 2; };
// FP64-accurate links and clover stored as float hi/lo pairs, double-float arithmetic
struct PDD { using T = dfloat; static constexpr int id = 3; };

// ---------------------------------------------------------------- geometry
struct Geom {
    int L[4];        // Lx, Ly, Lz, Lt
    int stride[4];   // 1, Lx, Lx*Ly, Lx*Ly*Lz
    int V;
    int antiperiodic;
};

DEV void site_coords(const Geom& g, int s, int c[4]) {
    c[0] = s % g.L[0];
    int r = s / g.L[0];
    c[1] = r % g.L[1];
    r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];
}
// neighbour x + dir*mu_hat; phase = -1 on an antiperiodic t wrap
DEV int neighbour(const Geom& g, int s, const int c[4], int mu, int dir, float& phase) {
    phase = 1.f;
    if (dir > 0) {
        if (c[mu] == g.L[mu] - 1) {
            if (mu == 3 && g.antiperiodic) phase = -1.f;
            return s - (g.L[mu] - 1) * g.stride[mu];
        }
        return s + g.stride[mu];
    } else {
        if (c[mu] == 0) {
            if (mu == 3 && g.antiperiodic) phase = -1.f;
            return s + (g.L[mu] - 1) * g.stride[mu];
        }
        return s - g.stride[mu];
    }
}

// Domain (multigrid block) geometry: block dims b, coarse dims C = L / b.
struct Blocking {
    int b[4];
    int C[4];
    int Vb;      // sites per block
    int Vc;      // number of blocks
};
// fine site of local index l in block Xi (both lexicographic, x fastest)
DEV int block_site(const Geom& g, const Blocking& bk, int Xi, int l, int c[4]) {
    int X[4], lc[4];
    X[0] = Xi % bk.C[0];
    int r = Xi / bk.C[0];
    X[1] = r % bk.C[1];
    r /= bk.C[1];
    X[2] = r % bk.C[2];
    X[3] = r / bk.C[2];
    lc[0] = l % bk.b[0];
    r = l / bk.b[0];
    lc[1] = r % bk.b[1];
    r /= bk.b[1];
    lc[2] = r % bk.b[2];
    lc[3] = r / bk.b[2];
    int s = 0;
    for (int mu = 3; mu >= 0; --mu) {
        c[mu] = X[mu] * bk.b[mu] + lc[mu];
    }
    s = c[0] + g.stride[1] * c[1] + g.stride[2] * c[2] + g.stride[3] * c[3];
    return s;
}

// ---------------------------------------------------------------- spinor storage
// Internal fine spinor layouts (per right-hand side, V sites):
//   P64: 12 chunks of double2  [k][V], k = spin*3 + colour
//   P32:  6 chunks of float4   [c][V], complex 2c in (x,y), 2c+1 in (z,w)
//   P16:  3 chunks of uint4    [c][V] (8 halves = 4 complex each) + float scale [V]
template <class P> struct SpinorIO;

template <> struct SpinorIO<P64> {
    static constexpr size_t bytes_per_site = 192;
    DEV static void load(const void* base, int V, int s, cx<double> v[12]) {
        const double2* p = (const double2*)base;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 t = __ldg(p + (size_t)k * V + s);
            v[k] = {t.x, t.y};
        }
    }
    DEV static void store(void* base, int V, int s, const cx<double> v[12]) {
        double2* p = (double2*)base;
#pragma unroll
        for (int k = 0; k < 12; ++k) p[(size_t)k * V + s] = make_double2(v[k].re, v[k].im);
    }
    // write only chirality half chi (complex components 6chi..6chi+5)
    DEV static void store_half(void* base, int V, int s, int chi, const cx<double> v[6]) {
        double2* p = (double2*)base + (size_t)6 * chi * V;
#pragma unroll
        for (int k = 0; k < 6; ++k) p[(size_t)k * V + s] = make_double2(v[k].re, v[k].im);
    }
    // plain (coherent) load for fields written by the same kernel launch
    DEV static void load_rw(const void* base, int V, int s, cx<double> v[12]) {
        const double2* p = (const double2*)base;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 t = p[(size_t)k * V + s];
            v[k] = {t.x, t.y};
        }
    }
};

template <> struct SpinorIO<P32> {
    static constexpr size_t bytes_per_site = 96;
    DEV static void load(const void* base, int V, int s, cx<float> v[12]) {
        const float4* p = (const float4*)base;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float4 t = __ldg(p + (size_t)c * V + s);
            v[2 * c] = {t.x, t.y};
            v[2 * c + 1] = {t.z, t.w};
        }
    }
    DEV static void store(void* base, int V, int s, const cx<float> v[12]) {
        float4* p = (float4*)base;
#pragma unroll
        for (int c = 0; c < 6; ++c)
            p[(size_t)c * V + s] = make_float4(v[2 * c].re, v[2 * c].im, v[2 * c + 1].re, v[2 * c + 1].im);
    }
    DEV static void store_half(void* base, int V, int s, int chi, const cx<float> v[6]) {
        float4* p = (float4*)base + (size_t)3 * chi * V;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            p[(size_t)c * V + s] = make_float4(v[2 * c].re, v[2 * c].im, v[2 * c + 1].re, v[2 * c + 1].im);
    }
    DEV static void load_rw(const void* base, int V, int s, cx<float> v[12]) {
        const float4* p = (const float4*)base;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float4 t = p[(size_t)c * V + s];
            v[2 * c] = {t.x, t.y};
            v[2 * c + 1] = {t.z, t.w};
        }
    }
};

// half spinor: the 48 bytes of halves are followed (after 3*V uint4) by V floats of scale
template <> struct SpinorIO<P16> {
    static constexpr size_t bytes_per_site = 52;
    DEV static void unpack(uint4 t, float sc, cx<float>* v) {
        const __half2* h = reinterpret_cast<const __half2*>(&t);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float2 f = __half22float2(h[q]);
            v[q] = {f.x * sc, f.y * sc};
        }
    }
    DEV static void load(const void* base, int V, int s, cx<float> v[12]) {
        const uint4* p = (const uint4*)base;
        const float* scale = (const float*)(p + (size_t)3 * V);
        float sc = __ldg(scale + s);
#pragma unroll
        for (int c = 0; c < 3; ++c) unpack(__ldg(p + (size_t)c * V + s), sc, v + 4 * c);
    }
    DEV static void load_rw(const void* base, int V, int s, cx<float> v[12]) {
        const uint4* p = (const uint4*)base;
        const float* scale = (const float*)(p + (size_t)3 * V);
        float sc = scale[s];
#pragma unroll
        for (int c = 0; c < 3; ++c) unpack(p[(size_t)c * V + s], sc, v + 4 * c);
    }
    DEV static void store(void* base, int V, int s, const cx<float> v[12]) {
        uint4* p = (uint4*)base;
        float* scale = (float*)(p + (size_t)3 * V);
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(v[k].re), fabsf(v[k].im)));
        float inv = m > 0.f ? 1.f / m : 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            uint4 t;
            __half2* h = reinterpret_cast<__half2*>(&t);
#pragma unroll
            for (int q = 0; q < 4; ++q) h[q] = __floats2half2_rn(v[4 * c + q].re * inv, v[4 * c + q].im * inv);
            p[(size_t)c * V + s] = t;
        }
        scale[s] = m;
    }
};

template <class P> HD size_t spinor_bytes(int V) { return SpinorIO<P>::bytes_per_site * (size_t)V; }

// ---------------------------------------------------------------- gauge storage
//   P64: [mu][9][V] double2 (full matrix, row-major)
//   P32: [mu][3][V] float4  (rows 0 and 1; row 2 = conj(row0 x row1))
//   P16: [mu][3][V] uint2   (rows 0 and 1 as halves)
template <typename T> DEV void reconstruct_row2(cx<T> u[3][3]) {
    cx<T> t0 = u[0][1] * u[1][2], t1 = u[0][2] * u[1][0], t2 = u[0][0] * u[1][1];
    cfma(t0, -u[0][2], u[1][1]);
    cfma(t1, -u[0][0], u[1][2]);
    cfma(t2, -u[0][1], u[1][0]);
    u[2][0] = conj(t0);
    u[2][1] = conj(t1);
    u[2][2] = conj(t2);
}

template <class P> struct GaugeIO;
template <> struct GaugeIO<P64> {
    static constexpr size_t bytes_per_link = 144;
    DEV static void load(const void* base, int V, int mu, int s, cx<double> u[3][3]) {
        const double2* p = (const double2*)base + (size_t)mu * 9 * V;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 t = __ldg(p + (size_t)k * V + s);
            u[k / 3][k % 3] = {t.x, t.y};
        }
    }
};
template <> struct GaugeIO<P32> {
    static constexpr size_t bytes_per_link = 48;
    DEV static void load(const void* base, int V, int mu, int s, cx<float> u[3][3]) {
        const float4* p = (const float4*)base + (size_t)mu * 3 * V;
        float4 a = __ldg(p + s), b = __ldg(p + (size_t)V + s), c = __ldg(p + (size_t)2 * V + s);
        u[0][0] = {a.x, a.y};
        u[0][1] = {a.z, a.w};
        u[0][2] = {b.x, b.y};
        u[1][0] = {b.z, b.w};
        u[1][1] = {c.x, c.y};
        u[1][2] = {c.z, c.w};
        reconstruct_row2(u);
    }
};
template <> struct GaugeIO<P16> {
    static constexpr size_t bytes_per_link = 24;
    DEV static void load(const void* base, int V, int mu, int s, cx<float> u[3][3]) {
        const uint2* p = (const uint2*)base + (size_t)mu * 3 * V;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            uint2 t = __ldg(p + (size_t)q * V + s);
            const __half2* h = reinterpret_cast<const __half2*>(&t);
            float2 f0 = __half22float2(h[0]), f1 = __half22float2(h[1]);
            int k0 = 2 * q, k1 = 2 * q + 1;
            u[k0 / 3][k0 % 3] = {f0.x, f0.y};
            u[k1 / 3][k1 % 3] = {f1.x, f1.y};
        }
        reconstruct_row2(u);
    }
};

// PDD: [mu][9][V] float4 = (re.hi, re.lo, im.hi, im.lo), full matrix
template <> struct GaugeIO<PDD> {
    static constexpr size_t bytes_per_link = 144;
    DEV static void load(const void* base, int V, int mu, int s, cx<dfloat> u[3][3]) {
        const float4* p = (const float4*)base + (size_t)mu * 9 * V;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float4 t = __ldg(p + (size_t)k * V + s);
            u[k / 3][k % 3] = {dfloat(t.x, t.y), dfloat(t.z, t.w)};
        }
    }
};

// ---------------------------------------------------------------- clover storage
// Two 6x6 Hermitian blocks per site (chirality 0: spins 0,1; 1: spins 2,3).
// Per block 18 real pairs: pairs 0..2 hold the six real diagonal entries,
// pairs 3..17 the strictly lower triangle L[i][j] (i > j) in row-major order,
// index 3 + i*(i-1)/2 + j.  Site layout: 36 pairs, block b at pairs 18b..18b+17.
//   P64: [36][V] double2;  P32: [18][V] float4 (pairs 2q, 2q+1);  P16: [9][V] uint4
template <class P> struct CloverIO;
template <> struct CloverIO<P64> {
    static constexpr size_t bytes_per_site = 576;
    DEV static void load_block(const void* base, int V, int s, int b, double pr[36]) {
        const double2* p = (const double2*)base + (size_t)18 * b * V;
#pragma unroll
        for (int q = 0; q < 18; ++q) {
            double2 t = __ldg(p + (size_t)q * V + s);
            pr[2 * q] = t.x;
            pr[2 * q + 1] = t.y;
        }
    }
};
template <> struct CloverIO<P32> {
    static constexpr size_t bytes_per_site = 288;
    DEV static void load_block(const void* base, int V, int s, int b, float pr[36]) {
        const float4* p = (const float4*)base + (size_t)9 * b * V;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            float4 t = __ldg(p + (size_t)q * V + s);
            pr[4 * q] = t.x;
            pr[4 * q + 1] = t.y;
            pr[4 * q + 2] = t.z;
            pr[4 * q + 3] = t.w;
        }
    }
};
template <> struct CloverIO<P16> {
    static constexpr size_t bytes_per_site = 144;
    DEV static void load_block(const void* base, int V, int s, int b, float pr[36]) {
        const uint4* p = (const uint4*)base;
        // 72 halves per site = 9 uint4; block 0 = halves 0..35, block 1 = 36..71
        // uint4 q holds halves 8q..8q+7
#pragma unroll
        for (int k = 0; k < 36; k += 2) {
            int hidx = 36 * b + k;
            uint4 t = __ldg(p + (size_t)(hidx / 8) * V + s);
            const __half2* h = reinterpret_cast<const __half2*>(&t);
            float2 f = __half22float2(h[(hidx % 8) / 2]);
            pr[k] = f.x;
            pr[k + 1] = f.y;
        }
    }
};

// PDD: [36][V] float4, pair q = (v0.hi, v0.lo, v1.hi, v1.lo)
template <> struct CloverIO<PDD> {
    static constexpr size_t bytes_per_site = 576;
    DEV static void load_block(const void* base, int V, int s, int b, dfloat pr[36]) {
        const float4* p = (const float4*)base + (size_t)18 * b * V;
#pragma unroll
        for (int q = 0; q < 18; ++q) {
            float4 t = __ldg(p + (size_t)q * V + s);
            pr[2 * q] = dfloat(t.x, t.y);
            pr[2 * q + 1] = dfloat(t.z, t.w);
        }
    }
};

// out[0..5] (+)= A_b in[0..5] for one Hermitian block in packed form
template <typename T> DEV void clover_block_apply(const T pr[36], const cx<T>* in, cx<T>* out) {
#pragma unroll
    for (int i = 0; i < 6; ++i) out[i] = pr[i] * in[i];
#pragma unroll
    for (int i = 1; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j < i; ++j) {
            int q = 3 + i * (i - 1) / 2 + j;
            cx<T> l = {pr[2 * q], pr[2 * q + 1]};
            cfma(out[i], l, in[j]);
            cfmac(out[j], l, in[i]);
        }
    }
}

template <class P>
DEV void clover_apply(const void* C, int V, int s, const cx<typename P::T> in[12], cx<typename P::T> out[12]) {
    using T = typename P::T;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        T pr[36];
        CloverIO<P>::load_block(C, V, s, b, pr);
        clover_block_apply<T>(pr, in + 6 * b, out + 6 * b);
    }
}

// ---------------------------------------------------------------- Wilson hop
// In the chiral basis gamma_mu = [[0, e_mu], [e_mu^dag, 0]] with e_k = i sigma_k
// (k = x, y, z) and e_t = 1.  For a spinor (u, l) in upper/lower spin pairs:
//   (1 - gamma_mu) psi = (h, -e_mu^dag h),  h = u - e_mu l
//   (1 + gamma_mu) psi = (h,  e_mu^dag h),  h = u + e_mu l
// so each hop multiplies only the half spinor h by the link.

// y = e_mu v for a spin pair (v0, v1) (one colour)
template <typename T> DEV void e_mul(int mu, cx<T> v0, cx<T> v1, cx<T>& y0, cx<T>& y1) {
    switch (mu) {
        case 0: y0 = timesI(v1); y1 = timesI(v0); break;          // i sigma_1
        case 1: y0 = v1; y1 = -v0; break;                          // i sigma_2
        case 2: y0 = timesI(v0); y1 = -timesI(v1); break;          // i sigma_3
        default: y0 = v0; y1 = v1; break;                          // 1
    }
}
// y = e_mu^dag v
template <typename T> DEV void edag_mul(int mu, cx<T> v0, cx<T> v1, cx<T>& y0, cx<T>& y1) {
    switch (mu) {
        case 0: y0 = -timesI(v1); y1 = -timesI(v0); break;
        case 1: y0 = -v1; y1 = v0; break;
        case 2: y0 = -timesI(v0); y1 = timesI(v1); break;
        default: y0 = v0; y1 = v1; break;
    }
}

// out += coeff * (1 - dir*gamma_mu) W psi, W = U (dir = +1) or U^dag (dir = -1)
template <typename T>
DEV void hop_accum(cx<T> out[12], const cx<T> psi[12], const cx<T> u[3][3], int mu, int dir, T coeff) {
    cx<T> h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<T> e0, e1;
        e_mul(mu, psi[6 + a], psi[9 + a], e0, e1);
        if (dir > 0) {
            h[0][a] = psi[a] - e0;
            h[1][a] = psi[3 + a] - e1;
        } else {
            h[0][a] = psi[a] + e0;
            h[1][a] = psi[3 + a] + e1;
        }
    }
    // W h for both spin components, then out_upper += coeff W h, out_lower -/+= coeff e^dag W h
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<T> w0, w1;
        if (dir > 0) {
            w0 = u[a][0] * h[0][0];
            w1 = u[a][0] * h[1][0];
            cfma(w0, u[a][1], h[0][1]);
            cfma(w1, u[a][1], h[1][1]);
            cfma(w0, u[a][2], h[0][2]);
            cfma(w1, u[a][2], h[1][2]);
        } else {
            w0 = cmulc(u[0][a], h[0][0]);
            w1 = cmulc(u[0][a], h[1][0]);
            cfmac(w0, u[1][a], h[0][1]);
            cfmac(w1, u[1][a], h[1][1]);
            cfmac(w0, u[2][a], h[0][2]);
            cfmac(w1, u[2][a], h[1][2]);
        }
        cx<T> l0, l1;
        edag_mul(mu, w0, w1, l0, l1);
        rfma(out[a], coeff, w0);
        rfma(out[3 + a], coeff, w1);
        const T cl = dir > 0 ? -coeff : coeff;
        rfma(out[6 + a], cl, l0);
        rfma(out[9 + a], cl, l1);
    }
}

// ---------------------------------------------------------------- reductions
template <typename T> DEV T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of NV values over the whole block; every thread gets the totals.
// scratch must hold NV * 32 values of T.  Contains two __syncthreads().
template <typename T, int NV>
DEV void block_sum(T (&v)[NV], T* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) scratch[k * 32 + warp] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        T t = T(0);
        for (int w = 0; w < nw; ++w) t += scratch[k * 32 + w];
        v[k] = t;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- ragged batches
// One problem of a ragged batch of independent solves (own lattice, operator
// and two-grid hierarchy), as the kernels of a fused phase read it: every
// phase is one launch whose CTAs are split among the problems by prefix
// offsets (off[p] .. off[p+1]-1 belong to problem p).  Filled on the host by
// ragged_dev_fill.  Precisions are fixed for the fused path: FP32 smoother
// and coarse vectors, FP64 outer vectors.
constexpr int kRaggedMaxBasis = 20;
struct RaggedDev {
    Geom g;
    Blocking bk;
    int nvec;
    float kappa32;
    double kappa;
    const void* U32;   // FP32 links, clover
    const void* C32;
    const void* Udd;   // double-float links, clover (FP64-accurate Arnoldi product)
    const void* Cdd;
    const void* vecs;  // test vectors (storage of the batch's vector precision)
    const void* v;     // V_j, FP64 internal
    void* f32;         // V_j in FP32
    void* f32b;        // FP32 scratch (the low part of x in the true residual)
    void* bc;          // coarse right-hand side, FP32 [Vc][2 nvec]
    void* xc;          // coarse solution
    void* z;           // Z_j = M V_j, FP32 internal
    void* w;           // D Z_j, FP64 internal
    const void* basis[kRaggedMaxBasis];   // V_0 .. V_j (flat FP64 complex)
    void* vnext;       // V_{j+1}
    double2* gs_part;  // Gram-Schmidt partials [quantity][n_blas]; the norm partials at gs_part + 2 R
    double2* gs_coef;  // [0..31] Hessenberg coefficients of pass 0, [32..] of pass 1, [63] |w'|
    size_t n;          // complex entries of a fine field
    size_t R;          // offset of the norm partials (in double2)
    // restart phases: true residual, its norm, V_0 = r / |r|, x += Z y, layout changes
    const void* U64;   // FP64 links, clover
    const void* C64;
    const void* b64;   // right-hand side, iterate, residual (FP64 internal)
    void* x64;
    void* r64;
    const void* rsrc;  // the vector whose norm is taken and normalised into basis[0]: r64, or b64 when x = 0
    double* npart;     // norm partials [n_blas]
    double* nval;      // its norm
    const void* zb[kRaggedMaxBasis];   // Z_0 .. Z_{k-1} (FP32 internal) and the coefficients y
    double2 yc[kRaggedMaxBasis];
    int k;
    const double* canon_in;   // canonical right-hand side and solution
    double* canon_out;
    int sap_nr;               // domains per CTA in the SAP half sweep (1 or 2)
};

// problem p and CTA index within it of this CTA for a prefix-offset table of np problems
DEV void ragged_locate(const int* __restrict__ off, int np, int& p, int& bx, int& gx) {
    int lo = 0, hi = np - 1;
    const int b = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    p = lo;
    bx = b - __ldg(off + lo);
    gx = __ldg(off + lo + 1) - __ldg(off + lo);
}
