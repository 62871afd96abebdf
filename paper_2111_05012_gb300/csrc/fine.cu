// Fine-lattice kernels: layout conversion, clover construction, the
// Wilson-clover stencil of Eq. 1 (full and domain-decomposed D_SAP) and the
// fused SAP half sweep (Sec. 3, SAP listing with minimal-residual domain
// solves).
#include <cstring>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kThreads = 256;

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
Blocking make_blocking(const GeomH& g, const BlockH& b) {
    Blocking k;
    k.Vb = 1;
    k.Vc = 1;
    for (int i = 0; i < 4; ++i) {
        k.b[i] = b.b[i];
        k.C[i] = g.L[i] / b.b[i];
        k.Vb *= k.b[i];
        k.Vc *= k.C[i];
    }
    return k;
}

int device_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}
int grid_for(int n, int threads) {
    const int sms = device_sms();
    int g = (n + threads - 1) / threads;
    int cap = sms * 16;
    return g < cap ? (g > 0 ? g : 1) : cap;
}

// ------------------------------------------------------------ pack / unpack
template <class P, typename E>
__global__ void pack_kernel(Geom g, const E* __restrict__ canon, void* internal, int nrhs) {
    using T = typename P::T;
    const int r = blockIdx.y;
    const E* src = canon + (size_t)r * g.V * 24;
    char* dst = (char*)internal + (size_t)r * spinor_bytes<P>(g.V);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        cx<T> v[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = {T(src[(size_t)s * 24 + 2 * k]), T(src[(size_t)s * 24 + 2 * k + 1])};
        SpinorIO<P>::store(dst, g.V, s, v);
    }
}
template <class P, typename E>
__global__ void unpack_kernel(Geom g, const void* internal, E* __restrict__ canon, int nrhs) {
    using T = typename P::T;
    const int r = blockIdx.y;
    E* dst = canon + (size_t)r * g.V * 24;
    const char* src = (const char*)internal + (size_t)r * spinor_bytes<P>(g.V);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        cx<T> v[12];
        SpinorIO<P>::load(src, g.V, s, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            dst[(size_t)s * 24 + 2 * k] = E(v[k].re);
            dst[(size_t)s * 24 + 2 * k + 1] = E(v[k].im);
        }
    }
}
// The same layout changes through a shared-memory tile of kTile sites: the canonical side of
// kTile consecutive sites is one contiguous block (24 values per site), read or written with
// 16-byte vector accesses by consecutive threads, while the internal side stays a coalesced
// per-site access (the per-site loops above leave each warp access spread over 32 sites'
// 192-byte records).  The tile pads each site's 24 values to 25 so that the per-site accesses
// of a warp fall in different banks.  Needs a 16-byte aligned canonical pointer.
constexpr int kTile = 128, kPad = 25;
template <typename E> struct Vec16;
template <> struct Vec16<double> {
    using T = double2;
    using E = double;
    static constexpr int n = 2;
    DEV static T make(const E* p) { return make_double2(p[0], p[1]); }
    DEV static void put(E* p, T v) { p[0] = v.x; p[1] = v.y; }
};
template <> struct Vec16<float> {
    using T = float4;
    static constexpr int n = 4;
    using E = float;
    DEV static T make(const E* p) { return make_float4(p[0], p[1], p[2], p[3]); }
    DEV static void put(E* p, T v) { p[0] = v.x; p[1] = v.y; p[2] = v.z; p[3] = v.w; }
};
// padded tile position of canonical element i of the tile (vectors never straddle a site)
DEV int tile_pos(int i) { return (i / 24) * kPad + i % 24; }

template <class P, typename E>
__global__ void __launch_bounds__(kTile) pack_tiled_kernel(Geom g, const E* __restrict__ canon, void* internal) {
    using T = typename P::T;
    using W = Vec16<E>;
    __shared__ E tile[kTile * kPad];
    const int r = blockIdx.y;
    const E* src = canon + (size_t)r * g.V * 24;
    char* dst = (char*)internal + (size_t)r * spinor_bytes<P>(g.V);
    for (int s0 = blockIdx.x * kTile; s0 < g.V; s0 += gridDim.x * kTile) {
        const int ns = min(kTile, g.V - s0);
        const typename W::T* vs = reinterpret_cast<const typename W::T*>(src + (size_t)s0 * 24);
        for (int i = threadIdx.x; i < ns * 24 / W::n; i += kTile) W::put(tile + tile_pos(i * W::n), vs[i]);
        __syncthreads();
        if (threadIdx.x < ns) {
            cx<T> v[12];
            const E* e = tile + threadIdx.x * kPad;
#pragma unroll
            for (int k = 0; k < 12; ++k) v[k] = {T(e[2 * k]), T(e[2 * k + 1])};
            SpinorIO<P>::store(dst, g.V, s0 + threadIdx.x, v);
        }
        __syncthreads();
    }
}
template <class P, typename E>
__global__ void __launch_bounds__(kTile) unpack_tiled_kernel(Geom g, const void* internal, E* __restrict__ canon) {
    using T = typename P::T;
    using W = Vec16<E>;
    __shared__ E tile[kTile * kPad];
    const int r = blockIdx.y;
    E* dst = canon + (size_t)r * g.V * 24;
    const char* src = (const char*)internal + (size_t)r * spinor_bytes<P>(g.V);
    for (int s0 = blockIdx.x * kTile; s0 < g.V; s0 += gridDim.x * kTile) {
        const int ns = min(kTile, g.V - s0);
        if (threadIdx.x < ns) {
            cx<T> v[12];
            SpinorIO<P>::load(src, g.V, s0 + threadIdx.x, v);
            E* e = tile + threadIdx.x * kPad;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                e[2 * k] = E(v[k].re);
                e[2 * k + 1] = E(v[k].im);
            }
        }
        __syncthreads();
        typename W::T* vd = reinterpret_cast<typename W::T*>(dst + (size_t)s0 * 24);
        for (int i = threadIdx.x; i < ns * 24 / W::n; i += kTile) vd[i] = W::make(tile + tile_pos(i * W::n));
        __syncthreads();
    }
}

template <class Pi, class Po>
__global__ void convert_kernel(Geom g, const void* in, void* out) {
    const int r = blockIdx.y;
    const char* src = (const char*)in + (size_t)r * spinor_bytes<Pi>(g.V);
    char* dst = (char*)out + (size_t)r * spinor_bytes<Po>(g.V);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        cx<typename Pi::T> v[12];
        cx<typename Po::T> w[12];
        SpinorIO<Pi>::load(src, g.V, s, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) w[k] = ccast<typename Po::T>(v[k]);
        SpinorIO<Po>::store(dst, g.V, s, w);
    }
}

// ------------------------------------------------------------ gauge
__global__ void gauge_convert_kernel(Geom g, const double* __restrict__ canon, void* out, int prec) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        for (int mu = 0; mu < 4; ++mu) {
            const double* m = canon + ((size_t)s * 4 + mu) * 18;
            if (prec == 0) {
                double2* p = (double2*)out + (size_t)mu * 9 * g.V;
                for (int k = 0; k < 9; ++k) p[(size_t)k * g.V + s] = make_double2(m[2 * k], m[2 * k + 1]);
            } else if (prec == 1) {
                float4* p = (float4*)out + (size_t)mu * 3 * g.V;
                for (int q = 0; q < 3; ++q)
                    p[(size_t)q * g.V + s] = make_float4((float)m[4 * q], (float)m[4 * q + 1], (float)m[4 * q + 2],
                                                         (float)m[4 * q + 3]);
            } else if (prec == 3) {
                float4* p = (float4*)out + (size_t)mu * 9 * g.V;
                for (int k = 0; k < 9; ++k) {
                    dfloat re = split_double(m[2 * k]), im = split_double(m[2 * k + 1]);
                    p[(size_t)k * g.V + s] = make_float4(re.hi, re.lo, im.hi, im.lo);
                }
            } else {
                uint2* p = (uint2*)out + (size_t)mu * 3 * g.V;
                for (int q = 0; q < 3; ++q) {
                    uint2 t;
                    __half2* h = reinterpret_cast<__half2*>(&t);
                    h[0] = __floats2half2_rn((float)m[4 * q], (float)m[4 * q + 1]);
                    h[1] = __floats2half2_rn((float)m[4 * q + 2], (float)m[4 * q + 3]);
                    p[(size_t)q * g.V + s] = t;
                }
            }
        }
    }
}

// ------------------------------------------------------------ clover
// sigma_munu restricted to the two chirality blocks: [plane][chirality][2][2]
__constant__ double2 c_sigma[6][2][2][2];

typedef cx<double> M3[3][3];

DEV void m3_mul(const M3 a, const M3 b, M3 c) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cx<double> t = czero<double>();
            for (int k = 0; k < 3; ++k) t = t + a[i][k] * b[k][j];
            c[i][j] = t;
        }
}
DEV void m3_dag(const M3 a, M3 c) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c[i][j] = conj(a[j][i]);
}
DEV int shifted(const Geom& g, const int c[4], int mu, int d, int nu, int e) {
    int cc[4] = {c[0], c[1], c[2], c[3]};
    cc[mu] = (cc[mu] + d + g.L[mu]) % g.L[mu];
    cc[nu] = (cc[nu] + e + g.L[nu]) % g.L[nu];
    return cc[0] + g.stride[1] * cc[1] + g.stride[2] * cc[2] + g.stride[3] * cc[3];
}
// product of four links a b c d (with optional daggers)
DEV void path4(const M3 a, const M3 b, const M3 c, const M3 d, M3 out) {
    M3 t1, t2;
    m3_mul(a, b, t1);
    m3_mul(t1, c, t2);
    m3_mul(t2, d, out);
}

// store the packed clover of one site (per chirality block: 6 real diagonal entries, then the
// 15 lower-triangle entries as (re, im) pairs) in the layout of precision P
template <class P>
DEV void clover_store(const double (&pr)[2][36], void* out, int V, int s) {
    if (P::id == 0) {
        double2* p = (double2*)out;
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < 18; ++q) p[(size_t)(18 * b + q) * V + s] = make_double2(pr[b][2 * q], pr[b][2 * q + 1]);
    } else if (P::id == 3) {
        float4* p = (float4*)out;
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < 18; ++q) {
                dfloat v0 = split_double(pr[b][2 * q]), v1 = split_double(pr[b][2 * q + 1]);
                p[(size_t)(18 * b + q) * V + s] = make_float4(v0.hi, v0.lo, v1.hi, v1.lo);
            }
    } else if (P::id == 1) {
        float4* p = (float4*)out;
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < 9; ++q)
                p[(size_t)(9 * b + q) * V + s] = make_float4((float)pr[b][4 * q], (float)pr[b][4 * q + 1],
                                                               (float)pr[b][4 * q + 2], (float)pr[b][4 * q + 3]);
    } else {
        uint4* p = (uint4*)out;
        for (int q = 0; q < 9; ++q) {
            uint4 t;
            __half2* h = reinterpret_cast<__half2*>(&t);
            for (int w = 0; w < 4; ++w) {
                int hidx = 8 * q + 2 * w;   // halves hidx, hidx+1 of the 72
                h[w] = __floats2half2_rn((float)pr[hidx / 36][hidx % 36], (float)pr[(hidx + 1) / 36][(hidx + 1) % 36]);
            }
            p[(size_t)q * V + s] = t;
        }
    }
}

template <class P>
__global__ void clover_build_kernel(Geom g, const void* U64, double kappa, double csw, void* out) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        int c[4];
        site_coords(g, s, c);
        cx<double> A[2][6][6];
        for (int b = 0; b < 2; ++b)
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) A[b][i][j] = czero<double>();
        int plane = 0;
        for (int mu = 0; mu < 4; ++mu) {
            for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
                M3 Q, L, u1, u2, u3, u4, d3, d4;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) Q[i][j] = czero<double>();
                // leaf x -> x+mu -> x+mu+nu -> x+nu -> x
                GaugeIO<P64>::load(U64, g.V, mu, s, u1);
                GaugeIO<P64>::load(U64, g.V, nu, shifted(g, c, mu, 1, nu, 0), u2);
                GaugeIO<P64>::load(U64, g.V, mu, shifted(g, c, mu, 0, nu, 1), u3);
                GaugeIO<P64>::load(U64, g.V, nu, s, u4);
                m3_dag(u3, d3);
                m3_dag(u4, d4);
                path4(u1, u2, d3, d4, L);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) Q[i][j] = Q[i][j] + L[i][j];
                // leaf x -> x+nu -> x+nu-mu -> x-mu -> x
                GaugeIO<P64>::load(U64, g.V, nu, s, u1);
                GaugeIO<P64>::load(U64, g.V, mu, shifted(g, c, mu, -1, nu, 1), u2);
                GaugeIO<P64>::load(U64, g.V, nu, shifted(g, c, mu, -1, nu, 0), u3);
                GaugeIO<P64>::load(U64, g.V, mu, shifted(g, c, mu, -1, nu, 0), u4);
                m3_dag(u2, d3);
                m3_dag(u3, d4);
                path4(u1, d3, d4, u4, L);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) Q[i][j] = Q[i][j] + L[i][j];
                // leaf x -> x-mu -> x-mu-nu -> x-nu -> x
                GaugeIO<P64>::load(U64, g.V, mu, shifted(g, c, mu, -1, nu, 0), u1);
                GaugeIO<P64>::load(U64, g.V, nu, shifted(g, c, mu, -1, nu, -1), u2);
                GaugeIO<P64>::load(U64, g.V, mu, shifted(g, c, mu, -1, nu, -1), u3);
                GaugeIO<P64>::load(U64, g.V, nu, shifted(g, c, mu, 0, nu, -1), u4);
                m3_dag(u1, d3);
                m3_dag(u2, d4);
                path4(d3, d4, u3, u4, L);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) Q[i][j] = Q[i][j] + L[i][j];
                // leaf x -> x-nu -> x-nu+mu -> x+mu -> x
                GaugeIO<P64>::load(U64, g.V, nu, shifted(g, c, mu, 0, nu, -1), u1);
                GaugeIO<P64>::load(U64, g.V, mu, shifted(g, c, mu, 0, nu, -1), u2);
                GaugeIO<P64>::load(U64, g.V, nu, shifted(g, c, mu, 1, nu, -1), u3);
                GaugeIO<P64>::load(U64, g.V, mu, s, u4);
                m3_dag(u1, d3);
                m3_dag(u4, d4);
                path4(d3, u2, u3, d4, L);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) Q[i][j] = Q[i][j] + L[i][j];
                // F = (Q - Q^dag) / (8i), traceless
                M3 F;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        cx<double> d = Q[i][j] - conj(Q[j][i]);
                        F[i][j] = {d.im / 8.0, -d.re / 8.0};   // d / (8i) = -i d / 8
                    }
                cx<double> tr = (1.0 / 3.0) * (F[0][0] + F[1][1] + F[2][2]);
                for (int i = 0; i < 3; ++i) F[i][i] = F[i][i] - tr;
                for (int b = 0; b < 2; ++b)
                    for (int al = 0; al < 2; ++al)
                        for (int be = 0; be < 2; ++be) {
                            double2 sg = c_sigma[plane][b][al][be];
                            cx<double> sgm = {-kappa * csw * sg.x, -kappa * csw * sg.y};
                            for (int a = 0; a < 3; ++a)
                                for (int bb = 0; bb < 3; ++bb)
                                    A[b][al * 3 + a][be * 3 + bb] = A[b][al * 3 + a][be * 3 + bb] + sgm * F[a][bb];
                        }
            }
        }
        // pack: 18 real pairs per block
        double pr[2][36];
        for (int b = 0; b < 2; ++b) {
            for (int i = 0; i < 6; ++i) pr[b][i] = 1.0 + A[b][i][i].re;
            for (int i = 1; i < 6; ++i)
                for (int j = 0; j < i; ++j) {
                    int q = 3 + i * (i - 1) / 2 + j;
                    pr[b][2 * q] = A[b][i][j].re;
                    pr[b][2 * q + 1] = A[b][i][j].im;
                }
        }
        clover_store<P>(pr, out, g.V, s);
    }
}

__global__ void clover_expand_kernel(Geom g, const void* C64, double* out) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        for (int b = 0; b < 2; ++b) {
            double pr[36];
            CloverIO<P64>::load_block(C64, g.V, s, b, pr);
            double* o = out + ((size_t)s * 2 + b) * 72;
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                    double re, im;
                    if (i == j) {
                        re = pr[i];
                        im = 0;
                    } else if (i > j) {
                        int q = 3 + i * (i - 1) / 2 + j;
                        re = pr[2 * q];
                        im = pr[2 * q + 1];
                    } else {
                        int q = 3 + j * (j - 1) / 2 + i;
                        re = pr[2 * q];
                        im = -pr[2 * q + 1];
                    }
                    o[(i * 6 + j) * 2] = re;
                    o[(i * 6 + j) * 2 + 1] = im;
                }
        }
    }
}

// ------------------------------------------------------------ Wilson-clover stencil
// FP32 / FP16: three CTAs per SM (the stencil streams from HBM and needs the
// warps); FP64: two (register cap 128)
template <class P, bool SAP, bool RESID>
DEV void dirac_site(const Geom& g, const Blocking& bk, const void* __restrict__ U, const void* __restrict__ C,
                    const char* src, char* dst, const char* bsrc, typename P::T kappa, int s) {
    using T = typename P::T;
    {
        int c[4];
        site_coords(g, s, c);
        cx<T> psi[12], acc[12];
        SpinorIO<P>::load(src, g.V, s, psi);
        clover_apply<P>(C, g.V, s, psi, acc);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            float ph;
            cx<T> u[3][3];
            if (!SAP || (c[mu] % bk.b[mu]) != bk.b[mu] - 1) {
                int n = neighbour(g, s, c, mu, +1, ph);
                SpinorIO<P>::load(src, g.V, n, psi);
                GaugeIO<P>::load(U, g.V, mu, s, u);
                hop_accum<T>(acc, psi, u, mu, +1, -kappa * T(ph));
            }
            if (!SAP || (c[mu] % bk.b[mu]) != 0) {
                int n = neighbour(g, s, c, mu, -1, ph);
                SpinorIO<P>::load(src, g.V, n, psi);
                GaugeIO<P>::load(U, g.V, mu, n, u);
                hop_accum<T>(acc, psi, u, mu, -1, -kappa * T(ph));
            }
        }
        if (RESID) {
            SpinorIO<P>::load(bsrc, g.V, s, psi);
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = psi[k] - acc[k];
        }
        SpinorIO<P>::store(dst, g.V, s, acc);
    }
}
// MB: resident CTAs per SM the register budget is set for (launch bounds; 0 = the default of
// the precision); the autotuner picks it with the CTA size and grid cap
template <class P, bool SAP, bool RESID, int MB = 0>
__global__ void __launch_bounds__(kThreads, MB ? MB : (P::id == 0 ? 2 : 3)) dirac_kernel(Geom g, Blocking bk, const void* __restrict__ U,
                                                         const void* __restrict__ C, const void* in, void* out,
                                                         const void* b, typename P::T kappa) {
    const int r = blockIdx.y;
    const size_t fb = spinor_bytes<P>(g.V);
    const char* src = (const char*)in + r * fb;
    char* dst = (char*)out + r * fb;
    const char* bsrc = RESID ? (const char*)b + r * fb : nullptr;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x)
        dirac_site<P, SAP, RESID>(g, bk, U, C, src, dst, bsrc, kappa, s);
}

// ragged batch, restart phases (site loops over each problem's lattice)
// r = b - D x with the FP64 stencil
__global__ void __launch_bounds__(kThreads, 2)
    resid64_ragged_kernel(const RaggedDev* __restrict__ d, const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    for (int s = bx * blockDim.x + threadIdx.x; s < q.g.V; s += gx * blockDim.x)
        dirac_site<P64, false, true>(q.g, q.bk, q.U64, q.C64, (const char*)q.x64, (char*)q.r64, (const char*)q.b64,
                                     q.kappa, s);
}
__global__ void pack_ragged_kernel(const RaggedDev* __restrict__ d, const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    for (int s = bx * blockDim.x + threadIdx.x; s < q.g.V; s += gx * blockDim.x) {
        cx<double> v[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = {q.canon_in[(size_t)s * 24 + 2 * k], q.canon_in[(size_t)s * 24 + 2 * k + 1]};
        SpinorIO<P64>::store(const_cast<void*>(q.b64), q.g.V, s, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = {0.0, 0.0};
        SpinorIO<P64>::store(q.x64, q.g.V, s, v);
    }
}
__global__ void unpack_ragged_kernel(const RaggedDev* __restrict__ d, const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    for (int s = bx * blockDim.x + threadIdx.x; s < q.g.V; s += gx * blockDim.x) {
        cx<double> v[12];
        SpinorIO<P64>::load(q.x64, q.g.V, s, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            q.canon_out[(size_t)s * 24 + 2 * k] = v[k].re;
            q.canon_out[(size_t)s * 24 + 2 * k + 1] = v[k].im;
        }
    }
}

// ------------------------------------------------------------ mixed stencil
// out (FP64) = D in for an FP32 input whose values are exact; links and
// clover are FP64 values held as float hi/lo pairs.  Every product of a
// float pair u = u_hi + u_lo with a float pair h = h_hi + h_lo is split
// into its exact leading part p = fl(u_hi h_hi) and a small correction
// (the FMA residual u_hi h_hi - p plus u_lo h_hi + u_hi h_lo); leading parts
// are summed with Knuth's two-sum (the rounding error of each addition is
// kept), corrections are summed in plain FP32.  The result carries about 46
// significant bits at roughly a third of the cost of full double-float
// arithmetic, and the work stays on the FP32 pipe.
struct fa {   // unevaluated sum hi + lo
    float hi, lo;
};
DEV fa fa_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
DEV void fa_add(fa& acc, fa v) {
    const fa t = fa_two_sum(acc.hi, v.hi);
    acc.hi = t.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t.lo, v.lo));
}
DEV fa fa_neg(fa v) { return {-v.hi, -v.lo}; }
// acc += u * h
DEV void fa_mac(fa& acc, dfloat u, fa h) {
    const float p = __fmul_rn(u.hi, h.hi);
    float e = fmaf(u.hi, h.hi, -p);
    e = fmaf(u.lo, h.hi, e);
    e = fmaf(u.hi, h.lo, e);
    const fa t = fa_two_sum(acc.hi, p);
    acc.hi = t.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t.lo, e));
}
// u * h as a pair (leading product and its correction)
DEV fa fa_mul(dfloat u, fa h) {
    const float p = __fmul_rn(u.hi, h.hi);
    float e = fmaf(u.hi, h.hi, -p);
    e = fmaf(u.lo, h.hi, e);
    e = fmaf(u.hi, h.lo, e);
    return {p, e};
}
struct cfa {
    fa re, im;
};
DEV cfa cfa_exact(cx<float> v) { return {{v.re, 0.f}, {v.im, 0.f}}; }
DEV void cfa_add(cfa& a, cfa b) {
    fa_add(a.re, b.re);
    fa_add(a.im, b.im);
}
// a += u h (conj(u) h when CONJ)
template <bool CONJ> DEV void cfa_mac(cfa& a, cx<dfloat> u, cfa h) {
    const dfloat ui = CONJ ? dfloat(-u.im.hi, -u.im.lo) : u.im;
    fa_mac(a.re, u.re, h.re);
    fa_mac(a.re, dfloat(-ui.hi, -ui.lo), h.im);
    fa_mac(a.im, u.re, h.im);
    fa_mac(a.im, ui, h.re);
}
// exact multiples: i v, -v
DEV cfa cfa_i(cfa v) { return {fa_neg(v.im), v.re}; }
DEV cfa cfa_neg(cfa v) { return {fa_neg(v.re), fa_neg(v.im)}; }
// y = e_mu v and y = e_mu^dag v for a spin pair (exact: signs and swaps)
DEV void cfa_e(int mu, cfa v0, cfa v1, cfa& y0, cfa& y1) {
    switch (mu) {
        case 0: y0 = cfa_i(v1); y1 = cfa_i(v0); break;
        case 1: y0 = v1; y1 = cfa_neg(v0); break;
        case 2: y0 = cfa_i(v0); y1 = cfa_neg(cfa_i(v1)); break;
        default: y0 = v0; y1 = v1; break;
    }
}
DEV void cfa_edag(int mu, cfa v0, cfa v1, cfa& y0, cfa& y1) {
    switch (mu) {
        case 0: y0 = cfa_neg(cfa_i(v1)); y1 = cfa_neg(cfa_i(v0)); break;
        case 1: y0 = cfa_neg(v1); y1 = v0; break;
        case 2: y0 = cfa_neg(cfa_i(v0)); y1 = cfa_i(v1); break;
        default: y0 = v0; y1 = v1; break;
    }
}
// sum of two exact-float complex values as an exact pair per component
DEV cfa cfa_sum(cfa a, cfa b) { return {fa_two_sum(a.re.hi, b.re.hi), fa_two_sum(a.im.hi, b.im.hi)}; }

// MODE 0: out(s) = (D in)(s) for one site s.
// MODE 1: out(s) = b(s) - (D (in + lo))(s) for an FP64 vector split into float parts in + lo
// (split_kernel): D in in the pair arithmetic, D lo in plain FP32 with the FP32 links and
// clover U32 / C32 (lo is 2^-24 of in or less, so FP32 rounding of that part stays below
// 2^-47 relative), its result the starting value of the pair accumulators.
// MODE 2: out(s) = (D (in + lo))(s), the same without b.
template <int MODE = 0>
DEV void dirac_mixed_site(const Geom& g, const void* __restrict__ U, const void* __restrict__ C, const char* src,
                          char* dst, dfloat kappa, int s, const void* __restrict__ U32 = nullptr,
                          const void* __restrict__ C32 = nullptr, const char* srclo = nullptr,
                          const char* bsrc = nullptr, float kappa32 = 0.f) {
    {
        int c[4];
        site_coords(g, s, c);
        cx<float> pf[12];
        cfa acc[12];
        if constexpr (MODE >= 1) {
            cx<float> lo[12];
            SpinorIO<P32>::load(srclo, g.V, s, pf);
            clover_apply<P32>(C32, g.V, s, pf, lo);
#pragma unroll 1
            for (int mu = 0; mu < 4; ++mu) {
                float ph;
                cx<float> u[3][3];
                int n = neighbour(g, s, c, mu, +1, ph);
                SpinorIO<P32>::load(srclo, g.V, n, pf);
                GaugeIO<P32>::load(U32, g.V, mu, s, u);
                hop_accum<float>(lo, pf, u, mu, +1, -kappa32 * ph);
                n = neighbour(g, s, c, mu, -1, ph);
                SpinorIO<P32>::load(srclo, g.V, n, pf);
                GaugeIO<P32>::load(U32, g.V, mu, n, u);
                hop_accum<float>(lo, pf, u, mu, -1, -kappa32 * ph);
            }
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = cfa_exact(lo[k]);
        }
        SpinorIO<P32>::load(src, g.V, s, pf);
        // clover: two packed Hermitian 6x6 blocks
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            dfloat pr[36];
            CloverIO<PDD>::load_block(C, g.V, s, b, pr);
            cfa* o = acc + 6 * b;
            const cx<float>* z = pf + 6 * b;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const cfa d = {fa_mul(pr[i], fa{z[i].re, 0.f}), fa_mul(pr[i], fa{z[i].im, 0.f})};
                if constexpr (MODE >= 1) cfa_add(o[i], d);
                else o[i] = d;
            }
#pragma unroll
            for (int i = 1; i < 6; ++i)
#pragma unroll
                for (int j = 0; j < i; ++j) {
                    const int q = 3 + i * (i - 1) / 2 + j;
                    const cx<dfloat> l = {pr[2 * q], pr[2 * q + 1]};
                    cfa_mac<false>(o[i], l, cfa_exact(z[j]));
                    cfa_mac<true>(o[j], l, cfa_exact(z[i]));
                }
        }
        // hops: h = (exact) projected half spinor, w = W h, out += -kappa * phase * (w, -/+ e^dag w);
        // the loop over the eight hops stays rolled: unrolled, the kernel body
        // does not fit the instruction cache
#pragma unroll 1
        for (int hop = 0; hop < 8; ++hop) {
            const int mu = hop >> 1, dir = (hop & 1) ? -1 : 1;
            {
                float ph;
                const int n = neighbour(g, s, c, mu, dir, ph);
                SpinorIO<P32>::load(src, g.V, n, pf);
                cx<dfloat> u[3][3];
                GaugeIO<PDD>::load(U, g.V, mu, dir > 0 ? s : n, u);
                const dfloat kc = dfloat(-ph * kappa.hi, -ph * kappa.lo);   // exact: ph = +-1
                cfa h[2][3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    cfa e0, e1;
                    cfa_e(mu, cfa_exact(pf[6 + a]), cfa_exact(pf[9 + a]), e0, e1);
                    if (dir < 0) {
                        h[0][a] = cfa_sum(cfa_exact(pf[a]), e0);
                        h[1][a] = cfa_sum(cfa_exact(pf[3 + a]), e1);
                    } else {
                        h[0][a] = cfa_sum(cfa_exact(pf[a]), cfa_neg(e0));
                        h[1][a] = cfa_sum(cfa_exact(pf[3 + a]), cfa_neg(e1));
                    }
                    // scale by -kappa * phase once, before the link
#pragma unroll
                    for (int sp = 0; sp < 2; ++sp)
                        h[sp][a] = {fa_mul(kc, h[sp][a].re), fa_mul(kc, h[sp][a].im)};
                }
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    cfa w0 = {{0.f, 0.f}, {0.f, 0.f}}, w1 = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        if (dir > 0) {
                            cfa_mac<false>(w0, u[a][b], h[0][b]);
                            cfa_mac<false>(w1, u[a][b], h[1][b]);
                        } else {
                            cfa_mac<true>(w0, u[b][a], h[0][b]);
                            cfa_mac<true>(w1, u[b][a], h[1][b]);
                        }
                    }
                    cfa l0, l1;
                    cfa_edag(mu, w0, w1, l0, l1);
                    cfa_add(acc[a], w0);
                    cfa_add(acc[3 + a], w1);
                    if (dir > 0) {
                        cfa_add(acc[6 + a], cfa_neg(l0));
                        cfa_add(acc[9 + a], cfa_neg(l1));
                    } else {
                        cfa_add(acc[6 + a], l0);
                        cfa_add(acc[9 + a], l1);
                    }
                }
            }
        }
        cx<double> o[12];
#pragma unroll
        for (int k = 0; k < 12; ++k)
            o[k] = {(double)acc[k].re.hi + (double)acc[k].re.lo, (double)acc[k].im.hi + (double)acc[k].im.lo};
        if constexpr (MODE == 1) {
            cx<double> bv[12];
            SpinorIO<P64>::load(bsrc, g.V, s, bv);
#pragma unroll
            for (int k = 0; k < 12; ++k) o[k] = bv[k] - o[k];
        }
        SpinorIO<P64>::store(dst, g.V, s, o);
    }
}

__global__ void __launch_bounds__(kThreads, 2) dirac_mixed_kernel(Geom g, const void* __restrict__ U,
                                                               const void* __restrict__ C, const void* in,
                                                               void* out, dfloat kappa) {
    const int r = blockIdx.y;
    const char* src = (const char*)in + r * spinor_bytes<P32>(g.V);
    char* dst = (char*)out + r * spinor_bytes<P64>(g.V);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x)
        dirac_mixed_site(g, U, C, src, dst, kappa, s);
}

// ragged batch: w = D z (FP32 z, FP64-accurate product) for every problem in one launch
__global__ void __launch_bounds__(kThreads, 2)
    dirac_mixed_ragged_kernel(const RaggedDev* __restrict__ d, const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    const dfloat kappa = split_double(q.kappa);
    for (int s = bx * blockDim.x + threadIdx.x; s < q.g.V; s += gx * blockDim.x)
        dirac_mixed_site(q.g, q.Udd, q.Cdd, (const char*)q.z, (char*)q.w, kappa, s);
}

// ragged batch: f32 = (float) v for every problem in one launch
__global__ void convert_ragged_kernel(const RaggedDev* __restrict__ d, const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    for (int s = bx * blockDim.x + threadIdx.x; s < q.g.V; s += gx * blockDim.x) {
        cx<double> v[12];
        cx<float> w[12];
        SpinorIO<P64>::load(q.v, q.g.V, s, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) w[k] = ccast<float>(v[k]);
        SpinorIO<P32>::store(q.f32, q.g.V, s, w);
    }
}

// ------------------------------------------------------------ FP64 vectors in the pair arithmetic
// D x (or b - D x) for FP64 x: x is first split into float parts hi + lo
// (split_kernel), then dirac_mixed_site<1> takes D hi in the pair arithmetic
// and D lo in plain FP32 (~46 significant bits; the outer solver's true
// residual on the FP32 pipe, FP64 arithmetic running at a small fraction of
// the FP32 rate here); the split is split_double_bits (integer and FP32
// instructions only).
__global__ void split_kernel(Geom g, const void* __restrict__ in, void* hi, void* lo) {
    const int r = blockIdx.y;
    const char* src = (const char*)in + r * spinor_bytes<P64>(g.V);
    char* dh = (char*)hi + r * spinor_bytes<P32>(g.V);
    char* dl = (char*)lo + r * spinor_bytes<P32>(g.V);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        cx<double> v[12];
        cx<float> h[12], l[12];
        SpinorIO<P64>::load(src, g.V, s, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const dfloat re = split_double_bits(v[k].re), im = split_double_bits(v[k].im);
            h[k] = {re.hi, im.hi};
            l[k] = {re.lo, im.lo};
        }
        SpinorIO<P32>::store(dh, g.V, s, h);
        SpinorIO<P32>::store(dl, g.V, s, l);
    }
}
template <bool RESID>
__global__ void __launch_bounds__(kThreads, 2)
    dirac_hilo_kernel(Geom g, const void* __restrict__ Udd, const void* __restrict__ Cdd,
                      const void* __restrict__ U32, const void* __restrict__ C32, const void* hi, const void* lo,
                      void* out, const void* b, dfloat kappa, float kappa32) {
    const int r = blockIdx.y;
    const char* sh = (const char*)hi + r * spinor_bytes<P32>(g.V);
    const char* sl = (const char*)lo + r * spinor_bytes<P32>(g.V);
    char* dst = (char*)out + r * spinor_bytes<P64>(g.V);
    const char* bs = RESID ? (const char*)b + r * spinor_bytes<P64>(g.V) : nullptr;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x)
        dirac_mixed_site<RESID ? 1 : 2>(g, Udd, Cdd, sh, dst, kappa, s, U32, C32, sl, bs, kappa32);
}

// ragged batch, true residual r = b - D x: x split into f32 (hi) and f32b (lo), then the pair stencil
__global__ void split_ragged_kernel(const RaggedDev* __restrict__ d, const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    for (int s = bx * blockDim.x + threadIdx.x; s < q.g.V; s += gx * blockDim.x) {
        cx<double> v[12];
        cx<float> h[12], l[12];
        SpinorIO<P64>::load(q.x64, q.g.V, s, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const dfloat re = split_double_bits(v[k].re), im = split_double_bits(v[k].im);
            h[k] = {re.hi, im.hi};
            l[k] = {re.lo, im.lo};
        }
        SpinorIO<P32>::store(q.f32, q.g.V, s, h);
        SpinorIO<P32>::store(q.f32b, q.g.V, s, l);
    }
}
__global__ void __launch_bounds__(kThreads, 2)
    resid_ragged_kernel(const RaggedDev* __restrict__ d, const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    const dfloat kappa = split_double(q.kappa);
    for (int s = bx * blockDim.x + threadIdx.x; s < q.g.V; s += gx * blockDim.x)
        dirac_mixed_site<1>(q.g, q.Udd, q.Cdd, (const char*)q.f32, (char*)q.r64, kappa, s, q.U32, q.C32,
                            (const char*)q.f32b, (const char*)q.b64, q.kappa32);
}

// x (FP64 internal) += sum_j c_j z_j for FP32 internal z_j: site by site,
// because the two internal layouts order the complex components differently
struct ZList {
    const void* p[20];
    double2 c[20];
};
__global__ void spinor_axpy_mixed_kernel(Geom g, int k, ZList z, void* x) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        cx<double> acc[12];
        SpinorIO<P64>::load_rw(x, g.V, s, acc);
        for (int j = 0; j < k; ++j) {
            cx<float> v[12];
            SpinorIO<P32>::load(z.p[j], g.V, s, v);
            const cx<double> cj = {z.c[j].x, z.c[j].y};
#pragma unroll
            for (int q = 0; q < 12; ++q) cfma(acc[q], cj, ccast<double>(v[q]));
        }
        SpinorIO<P64>::store(x, g.V, s, acc);
    }
}

// the same in pair arithmetic on the FP32 pipe: x split into float pairs (split_double_bits),
// c_j split likewise, the products with the exact floats of z_j and the sums kept as pairs,
// one FP64 addition per stored value
DEV void pmac_exact(dfloat& a, dfloat c, float z) {
    const float p = __fmul_rn(c.hi, z);
    float e = fmaf(c.hi, z, -p);
    e = fmaf(c.lo, z, e);
    const dfloat t = two_sum(a.hi, p);
    a.hi = t.hi;
    a.lo = __fadd_rn(a.lo, __fadd_rn(t.lo, e));
}
__global__ void spinor_axpy_mixed_df_kernel(Geom g, int k, ZList z, void* x) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        cx<double> acc[12];
        SpinorIO<P64>::load_rw(x, g.V, s, acc);
        dfloat ar[12], ai[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            ar[q] = split_double_bits(acc[q].re);
            ai[q] = split_double_bits(acc[q].im);
        }
        for (int j = 0; j < k; ++j) {
            cx<float> v[12];
            SpinorIO<P32>::load(z.p[j], g.V, s, v);
            const dfloat cr = split_double_bits(z.c[j].x), ci = split_double_bits(z.c[j].y);
            const dfloat nci(-ci.hi, -ci.lo);
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                pmac_exact(ar[q], cr, v[q].re);
                pmac_exact(ar[q], nci, v[q].im);
                pmac_exact(ai[q], cr, v[q].im);
                pmac_exact(ai[q], ci, v[q].re);
            }
        }
#pragma unroll
        for (int q = 0; q < 12; ++q) acc[q] = {pair_to_double(ar[q].hi, ar[q].lo), pair_to_double(ai[q].hi, ai[q].lo)};
        SpinorIO<P64>::store(x, g.V, s, acc);
    }
}

// ragged batch: x64 += sum_{i<k} yc_i Z_i for every problem (k and y per problem)
__global__ void xupdate_ragged_kernel(const RaggedDev* __restrict__ d, const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    for (int s = bx * blockDim.x + threadIdx.x; s < q.g.V; s += gx * blockDim.x) {
        cx<double> acc[12];
        SpinorIO<P64>::load_rw(q.x64, q.g.V, s, acc);
        for (int j = 0; j < q.k; ++j) {
            cx<float> v[12];
            SpinorIO<P32>::load(q.zb[j], q.g.V, s, v);
            const cx<double> cj = {q.yc[j].x, q.yc[j].y};
#pragma unroll
            for (int t = 0; t < 12; ++t) cfma(acc[t], cj, ccast<double>(v[t]));
        }
        SpinorIO<P64>::store(q.x64, q.g.V, s, acc);
    }
}

// ------------------------------------------------------------ domain vector in shared memory
// The residual of a domain, one site per thread: FP32 as [6][vbp] float4 (two
// complex numbers per 16-byte access), FP64 as [12][vbp] complex; 96 / 192
// bytes per site either way.
template <typename T> struct DomainVec;
template <> struct DomainVec<float> {
    DEV static void put(void* sh, int vbp, int l, const cx<float> v[12]) {
        float4* p = (float4*)sh;
#pragma unroll
        for (int c = 0; c < 6; ++c) p[c * vbp + l] = make_float4(v[2 * c].re, v[2 * c].im, v[2 * c + 1].re, v[2 * c + 1].im);
    }
    DEV static void get(const void* sh, int vbp, int l, cx<float> v[12]) {
        const float4* p = (const float4*)sh;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float4 t = p[c * vbp + l];
            v[2 * c] = {t.x, t.y};
            v[2 * c + 1] = {t.z, t.w};
        }
    }
};
template <> struct DomainVec<double> {
    DEV static void put(void* sh, int vbp, int l, const cx<double> v[12]) {
        cx<double>* p = (cx<double>*)sh;
#pragma unroll
        for (int q = 0; q < 12; ++q) p[q * vbp + l] = v[q];
    }
    DEV static void get(const void* sh, int vbp, int l, cx<double> v[12]) {
        const cx<double>* p = (const cx<double>*)sh;
#pragma unroll
        for (int q = 0; q < 12; ++q) v[q] = p[q * vbp + l];
    }
};

// A^{-1} per site from the FP64 clover (A = 1 + F: two Hermitian 6x6 blocks, each inverted
// by Gauss-Jordan elimination with partial pivoting in FP64; the inverse is Hermitian and is
// stored in the clover's packed form, from the mean of its lower and conjugated upper triangle)
template <class P>
__global__ void clover_invert_kernel(Geom g, const void* C64, void* out) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        double pr[2][36];
        const double2* src = (const double2*)C64;
        for (int b = 0; b < 2; ++b) {
            for (int q = 0; q < 18; ++q) {
                double2 t = src[(size_t)(18 * b + q) * g.V + s];
                pr[b][2 * q] = t.x;
                pr[b][2 * q + 1] = t.y;
            }
            cx<double> M[6][6], R[6][6];
            for (int i = 0; i < 6; ++i) {
                M[i][i] = {pr[b][i], 0.0};
                for (int j = 0; j < i; ++j) {
                    const int q = 3 + i * (i - 1) / 2 + j;
                    M[i][j] = {pr[b][2 * q], pr[b][2 * q + 1]};
                    M[j][i] = conj(M[i][j]);
                }
                for (int j = 0; j < 6; ++j) R[i][j] = {i == j ? 1.0 : 0.0, 0.0};
            }
            for (int c = 0; c < 6; ++c) {
                int piv = c;
                double best = norm2(M[c][c]);
                for (int i = c + 1; i < 6; ++i)
                    if (norm2(M[i][c]) > best) {
                        best = norm2(M[i][c]);
                        piv = i;
                    }
                if (piv != c)
                    for (int j = 0; j < 6; ++j) {
                        cx<double> t = M[c][j];
                        M[c][j] = M[piv][j];
                        M[piv][j] = t;
                        t = R[c][j];
                        R[c][j] = R[piv][j];
                        R[piv][j] = t;
                    }
                const cx<double> d = M[c][c];
                const double dn = norm2(d);
                const cx<double> inv = {d.re / dn, -d.im / dn};
                for (int j = 0; j < 6; ++j) {
                    M[c][j] = inv * M[c][j];
                    R[c][j] = inv * R[c][j];
                }
                for (int i = 0; i < 6; ++i) {
                    if (i == c) continue;
                    const cx<double> f = M[i][c];
                    for (int j = 0; j < 6; ++j) {
                        M[i][j] = M[i][j] - f * M[c][j];
                        R[i][j] = R[i][j] - f * R[c][j];
                    }
                }
            }
            for (int i = 0; i < 6; ++i) {
                pr[b][i] = R[i][i].re;
                for (int j = 0; j < i; ++j) {
                    const int q = 3 + i * (i - 1) / 2 + j;
                    const cx<double> h = 0.5 * (R[i][j] + conj(R[j][i]));
                    pr[b][2 * q] = h.re;
                    pr[b][2 * q + 1] = h.im;
                }
            }
        }
        clover_store<P>(pr, out, g.V, s);
    }
}

// ------------------------------------------------------------ SAP half sweep
// One CTA per domain of the given colour, one thread per site of the domain.
// Computes r = b - D x on the domain (the residual of the SAP listing, needed
// only where the next inner solve reads it), runs nmr minimal-residual steps
// on D_SAP restricted to the domain with r kept in shared memory, and adds the
// result to x.  Domains of one colour never touch each other (even number of
// domains per direction), so the CTAs are independent.
// x_mode: 0 = x holds the current iterate everywhere; 1 = x is zero everywhere
// (r = b, x is only written); 2 = x is zero on the active domains and holds the
// iterate elsewhere (first odd half sweep after an even sweep from zero).
// 256-thread FP32/FP16 variant: 128 registers, two CTAs per SM (no spills);
// the FP64 variant keeps one CTA per SM (it would spill at 128 registers)
// NR right-hand sides per CTA (NR = 2 for batches, variant 2): thread (slot, l) works on site l
// for right-hand side NR * (pair index) + slot; both slots read the same domain's links and
// clover in lockstep, so one domain's operator occupies the SM's L1 instead of two domains'.
// The body of one CTA: domain k of the given colour, right-hand sides NR * rpair + slot; with
// DS the NR slots take domains NR * k + slot of right-hand side rpair instead (small domains
// of a ragged batch, two to a CTA)
template <class P, int NR, bool DS = false>
DEV void sap_half_body(const Geom& g, const Blocking& bk, int colour, int nmr, int x_mode,
                       const void* __restrict__ U, const void* __restrict__ C, const void* __restrict__ b, void* x,
                       typename P::T kappa, int k0, int rpair, int nrhs) {
    using T = typename P::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int vbp = blockDim.x / NR;
    const int slot = NR == 1 ? 0 : threadIdx.x / vbp;
    cx<T>* rsh = reinterpret_cast<cx<T>*>(smem_raw) + (size_t)slot * 12 * vbp;      // [NR][12][vbp]
    T* red = reinterpret_cast<T*>(reinterpret_cast<cx<T>*>(smem_raw) + (size_t)NR * 12 * vbp) + slot * 192;   // [NR][2][3][32]
    const int rr = DS ? rpair : NR * rpair + slot;
    const int k = DS ? NR * k0 + slot : k0;
    const bool rhs_ok = rr < nrhs && (!DS || k < bk.Vc / 2);
    const int h0 = bk.C[0] / 2;
    int rest = k / h0;
    int X1 = rest % bk.C[1];
    rest /= bk.C[1];
    int X2 = rest % bk.C[2];
    int X3 = rest / bk.C[2];
    int X0 = 2 * (k % h0) + ((X1 + X2 + X3 + colour) & 1);
    const int Xi = X0 + bk.C[0] * (X1 + bk.C[1] * (X2 + bk.C[2] * X3));

    const int l = threadIdx.x - slot * vbp;
    const bool active = l < bk.Vb && rhs_ok;
    int c[4] = {0, 0, 0, 0}, lc[4] = {0, 0, 0, 0}, s = 0;
    const int lstr[4] = {1, bk.b[0], bk.b[0] * bk.b[1], bk.b[0] * bk.b[1] * bk.b[2]};
    cx<T> r[12], z[12], Ar[12];
    b = (const char*)b + (rhs_ok ? rr : 0) * spinor_bytes<P>(g.V);
    x = (char*)x + (rhs_ok ? rr : 0) * spinor_bytes<P>(g.V);
    if (active) {
        s = block_site(g, bk, Xi, l, c);
        for (int mu = 0; mu < 4; ++mu) lc[mu] = c[mu] % bk.b[mu];
        SpinorIO<P>::load(b, g.V, s, r);
        if (x_mode != 1) {
            // r = b - D x at this site; with x_mode 2 only hops from outside the domain contribute
            cx<T> psi[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) Ar[q] = czero<T>();
            if (x_mode == 0) {
                SpinorIO<P>::load(x, g.V, s, psi);
                clover_apply<P>(C, g.V, s, psi, Ar);
            }
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                float ph;
                cx<T> u[3][3];
                if (x_mode == 0 || lc[mu] == bk.b[mu] - 1) {
                    int n = neighbour(g, s, c, mu, +1, ph);
                    SpinorIO<P>::load(x, g.V, n, psi);
                    GaugeIO<P>::load(U, g.V, mu, s, u);
                    hop_accum<T>(Ar, psi, u, mu, +1, -kappa * T(ph));
                }
                if (x_mode == 0 || lc[mu] == 0) {
                    int n = neighbour(g, s, c, mu, -1, ph);
                    SpinorIO<P>::load(x, g.V, n, psi);
                    GaugeIO<P>::load(U, g.V, mu, n, u);
                    hop_accum<T>(Ar, psi, u, mu, -1, -kappa * T(ph));
                }
            }
#pragma unroll
            for (int q = 0; q < 12; ++q) r[q] = r[q] - Ar[q];
        }
#pragma unroll
        for (int q = 0; q < 12; ++q) z[q] = czero<T>();
        DomainVec<T>::put(rsh, vbp, l, r);
    }
    for (int it = 0; it < nmr; ++it) {
        __syncthreads();
        T part[3] = {T(0), T(0), T(0)};
        if (active) {
            clover_apply<P>(C, g.V, s, r, Ar);
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                cx<T> u[3][3], psi[12];
                if (lc[mu] != bk.b[mu] - 1) {
                    DomainVec<T>::get(rsh, vbp, l + lstr[mu], psi);
                    GaugeIO<P>::load(U, g.V, mu, s, u);
                    hop_accum<T>(Ar, psi, u, mu, +1, -kappa);
                }
                if (lc[mu] != 0) {
                    DomainVec<T>::get(rsh, vbp, l - lstr[mu], psi);
                    GaugeIO<P>::load(U, g.V, mu, s - g.stride[mu], u);
                    hop_accum<T>(Ar, psi, u, mu, -1, -kappa);
                }
            }
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                // <Ar, r> and |Ar|^2 as fused multiply-adds
                part[0] = fma(Ar[q].re, r[q].re, part[0]);
                part[0] = fma(Ar[q].im, r[q].im, part[0]);
                part[1] = fma(Ar[q].re, r[q].im, part[1]);
                part[1] = fma(-Ar[q].im, r[q].re, part[1]);
                part[2] = fma(Ar[q].re, Ar[q].re, part[2]);
                part[2] = fma(Ar[q].im, Ar[q].im, part[2]);
            }
        }
        // one-barrier block reduction into buffer (it & 1): the loop's top barrier keeps the
        // other buffer's readers of the previous step apart from its next writers
        {
            const int lane = l & 31, warp = l >> 5, nw = (vbp + 31) >> 5;
            T* rb = red + (it & 1) * 96;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                T v = warp_sum(part[q]);
                if (lane == 0) rb[q * 32 + warp] = v;
            }
            __syncthreads();
            part[0] = part[1] = part[2] = T(0);
            for (int w = 0; w < nw; ++w) {
                part[0] += rb[w];
                part[1] += rb[32 + w];
                part[2] += rb[64 + w];
            }
        }
        cx<T> alpha = czero<T>();
        if (part[2] > T(0)) alpha = {part[0] / part[2], part[1] / part[2]};
        if (active) {
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                cfma(z[q], alpha, r[q]);
                cfma(r[q], -alpha, Ar[q]);
            }
            DomainVec<T>::put(rsh, vbp, l, r);
        }
    }
    if (active) {
        if (x_mode == 0) {
            cx<T> x0[12];
            SpinorIO<P>::load(x, g.V, s, x0);
#pragma unroll
            for (int q = 0; q < 12; ++q) z[q] = z[q] + x0[q];
        }
        SpinorIO<P>::store(x, g.V, s, z);
    }
}

// domain of a CTA: the k-th domain of the given colour; right-hand side group of a batch.
// rhs_fast: the right-hand side is the fast grid index, so the CTAs of one domain for all
// right-hand sides run together and share the domain's links and clover in L1/L2
template <class P, int MAXT, int NR>
__global__ void __launch_bounds__(MAXT * NR, (MAXT == 256 && NR == 1 && P::id != 0) ? 2 : 1)
    sap_half_kernel(Geom g, Blocking bk, int colour, int nmr, int x_mode, const void* __restrict__ U,
                    const void* __restrict__ C, const void* __restrict__ b, void* x, typename P::T kappa,
                    int rhs_fast, int nrhs) {
    sap_half_body<P, NR>(g, bk, colour, nmr, x_mode, U, C, b, x, kappa, rhs_fast ? blockIdx.y : blockIdx.x,
                         rhs_fast ? blockIdx.x : blockIdx.y, nrhs);
}

// the half sweep for every problem of a ragged batch in one launch: CTA ranges per problem
// from the prefix table off (the problem's domains of this colour, sap_nr to a CTA), FP32,
// right-hand side V_j in f32, iterate Z_j in z.  blockDim covers the largest domain; a
// problem whose domains fit half of it takes two domains per CTA (sap_nr = 2)
__global__ void __launch_bounds__(256, 2)
    sap_half_ragged_kernel(const RaggedDev* __restrict__ d, const int* __restrict__ off, int np, int colour,
                           int nmr) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    if (q.sap_nr == 2) sap_half_body<P32, 2, true>(q.g, q.bk, colour, nmr, 0, q.U32, q.C32, q.f32, q.z, q.kappa32, bx, 0, 1);
    else sap_half_body<P32, 1>(q.g, q.bk, colour, nmr, 0, q.U32, q.C32, q.f32, q.z, q.kappa32, bx, 0, 1);
}

// ------------------------------------------------------------ SAP half sweep, even-odd domain solves
// The half sweep of sap_half_kernel with each domain solve in Schur-complement
// form (reading C28): with the domain operator split by site parity,
// D_SAP = [[A_ee, H_eo], [H_oe, A_oo]] (H the in-domain hops, A = 1 + F),
//   rho = r_e - H_eo A_oo^{-1} r_o,  nmr minimal-residual steps on
//   S = A_ee - H_eo A_oo^{-1} H_oe from z_e = 0,  z_o = A_oo^{-1} (r_o - H_oe z_e).
// One CTA per domain of the given colour, one thread per pair of x-neighbouring
// sites (one even, one odd: the block's x extent is even), so both parity
// phases of a step keep every warp busy.  The domain tile of shared memory
// holds rho (later z) on even sites and A_oo^{-1} H_oe rho on odd sites; the
// odd sites' residual r_o waits in a second tile for the reconstruction.
template <class P>
__global__ void __launch_bounds__(128, P::id == 0 ? 2 : 4)
    sap_half_eo_kernel(Geom g, Blocking bk, int colour, int nmr, int x_mode, const void* __restrict__ U,
                       const void* __restrict__ C, const void* __restrict__ Ci, const void* __restrict__ b, void* x,
                       typename P::T kappa, int rhs_fast) {
    using T = typename P::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int vbp = 2 * blockDim.x;                           // domain sites (padded)
    cx<T>* sh = reinterpret_cast<cx<T>*>(smem_raw);          // [12][vbp] by domain site
    cx<T>* ros = sh + 12 * vbp;                               // [12][blockDim.x] r_o of each pair
    T* red = reinterpret_cast<T*>(ros + 12 * blockDim.x);     // [3][32]

    const int k = rhs_fast ? blockIdx.y : blockIdx.x;
    const int rr = rhs_fast ? blockIdx.x : blockIdx.y;
    const int h0 = bk.C[0] / 2;
    int rest = k / h0;
    int X1 = rest % bk.C[1];
    rest /= bk.C[1];
    int X2 = rest % bk.C[2];
    int X3 = rest / bk.C[2];
    int X0 = 2 * (k % h0) + ((X1 + X2 + X3 + colour) & 1);
    const int Xi = X0 + bk.C[0] * (X1 + bk.C[1] * (X2 + bk.C[2] * X3));
    b = (const char*)b + rr * spinor_bytes<P>(g.V);
    x = (char*)x + rr * spinor_bytes<P>(g.V);

    const int t = threadIdx.x;
    const bool active = 2 * t < bk.Vb;
    const int lstr[4] = {1, bk.b[0], bk.b[0] * bk.b[1], bk.b[0] * bk.b[1] * bk.b[2]};
    // the pair's sites: domain indices le (even parity) and lo (odd), global sites se, so
    int le = 0, lo = 0, se = 0, so = 0, ce[4] = {0, 0, 0, 0}, co[4] = {0, 0, 0, 0}, lce[4], lco[4];
    if (active) {
        int c0[4], c1[4];
        const int s0 = block_site(g, bk, Xi, 2 * t, c0);
        const int s1 = block_site(g, bk, Xi, 2 * t + 1, c1);
        const bool first_even = ((c0[0] + c0[1] + c0[2] + c0[3]) & 1) == 0;
        le = first_even ? 2 * t : 2 * t + 1;
        lo = first_even ? 2 * t + 1 : 2 * t;
        se = first_even ? s0 : s1;
        so = first_even ? s1 : s0;
        for (int mu = 0; mu < 4; ++mu) {
            ce[mu] = first_even ? c0[mu] : c1[mu];
            co[mu] = first_even ? c1[mu] : c0[mu];
            lce[mu] = ce[mu] % bk.b[mu];
            lco[mu] = co[mu] % bk.b[mu];
        }
    }
    // r = b - D x at one site (hops may leave the domain; x_mode as in sap_half_kernel)
    auto residual = [&](int s, const int (&c)[4], const int (&lc)[4], cx<T> (&r)[12]) {
        SpinorIO<P>::load(b, g.V, s, r);
        if (x_mode == 1) return;
        cx<T> psi[12], acc[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) acc[q] = czero<T>();
        if (x_mode == 0) {
            SpinorIO<P>::load(x, g.V, s, psi);
            clover_apply<P>(C, g.V, s, psi, acc);
        }
        int cc[4] = {c[0], c[1], c[2], c[3]};
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            float ph;
            cx<T> u[3][3];
            if (x_mode == 0 || lc[mu] == bk.b[mu] - 1) {
                int n = neighbour(g, s, cc, mu, +1, ph);
                SpinorIO<P>::load(x, g.V, n, psi);
                GaugeIO<P>::load(U, g.V, mu, s, u);
                hop_accum<T>(acc, psi, u, mu, +1, -kappa * T(ph));
            }
            if (x_mode == 0 || lc[mu] == 0) {
                int n = neighbour(g, s, cc, mu, -1, ph);
                SpinorIO<P>::load(x, g.V, n, psi);
                GaugeIO<P>::load(U, g.V, mu, n, u);
                hop_accum<T>(acc, psi, u, mu, -1, -kappa * T(ph));
            }
        }
#pragma unroll
        for (int q = 0; q < 12; ++q) r[q] = r[q] - acc[q];
    };
    // acc += coeff * (in-domain hops of site s from the tile)
    auto tile_hops = [&](int s, int l, const int (&lc)[4], T coeff, cx<T> (&acc)[12]) {
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            cx<T> u[3][3], psi[12];
            if (lc[mu] != bk.b[mu] - 1) {
                DomainVec<T>::get(sh, vbp, l + lstr[mu], psi);
                GaugeIO<P>::load(U, g.V, mu, s, u);
                hop_accum<T>(acc, psi, u, mu, +1, coeff);
            }
            if (lc[mu] != 0) {
                DomainVec<T>::get(sh, vbp, l - lstr[mu], psi);
                GaugeIO<P>::load(U, g.V, mu, s - g.stride[mu], u);
                hop_accum<T>(acc, psi, u, mu, -1, coeff);
            }
        }
    };
    cx<T> rho[12], z[12], v[12];
    if (active) {
        // r_o -> A_oo^{-1} r_o in the tile; r_o kept for the reconstruction
        residual(so, co, lco, v);
        DomainVec<T>::put(ros, blockDim.x, t, v);
        cx<T> w[12];
        clover_apply<P>(Ci, g.V, so, v, w);
        DomainVec<T>::put(sh, vbp, lo, w);
        residual(se, ce, lce, rho);
    }
    __syncthreads();
    if (active) {
        // rho = r_e - H_eo A_oo^{-1} r_o  (H = -kappa * hop terms)
        tile_hops(se, le, lce, kappa, rho);
#pragma unroll
        for (int q = 0; q < 12; ++q) z[q] = czero<T>();
    }
    for (int it = 0; it < nmr; ++it) {
        if (active) DomainVec<T>::put(sh, vbp, le, rho);
        __syncthreads();
        // odd sites: w = A_oo^{-1} H_oe rho
        if (active) {
#pragma unroll
            for (int q = 0; q < 12; ++q) v[q] = czero<T>();
            tile_hops(so, lo, lco, -kappa, v);
            cx<T> w[12];
            clover_apply<P>(Ci, g.V, so, v, w);
            DomainVec<T>::put(sh, vbp, lo, w);
        }
        __syncthreads();
        // even sites: S rho = A_ee rho - H_eo w
        T part[3] = {T(0), T(0), T(0)};
        if (active) {
            clover_apply<P>(C, g.V, se, rho, v);
            tile_hops(se, le, lce, kappa, v);
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                part[0] = fma(v[q].re, rho[q].re, part[0]);
                part[0] = fma(v[q].im, rho[q].im, part[0]);
                part[1] = fma(v[q].re, rho[q].im, part[1]);
                part[1] = fma(-v[q].im, rho[q].re, part[1]);
                part[2] = fma(v[q].re, v[q].re, part[2]);
                part[2] = fma(v[q].im, v[q].im, part[2]);
            }
        }
        block_sum<T, 3>(part, red);
        cx<T> alpha = czero<T>();
        if (part[2] > T(0)) alpha = {part[0] / part[2], part[1] / part[2]};
        if (active) {
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                cfma(z[q], alpha, rho[q]);
                cfma(rho[q], -alpha, v[q]);
            }
        }
    }
    // z_o = A_oo^{-1} (r_o - H_oe z_e), then x += z on both sites
    if (active) DomainVec<T>::put(sh, vbp, le, z);
    __syncthreads();
    if (active) {
        DomainVec<T>::get(ros, blockDim.x, t, v);
        tile_hops(so, lo, lco, kappa, v);
        cx<T> zo[12];
        clover_apply<P>(Ci, g.V, so, v, zo);
        if (x_mode == 0) {
            cx<T> x0[12];
            SpinorIO<P>::load(x, g.V, se, x0);
#pragma unroll
            for (int q = 0; q < 12; ++q) z[q] = z[q] + x0[q];
            SpinorIO<P>::load(x, g.V, so, x0);
#pragma unroll
            for (int q = 0; q < 12; ++q) zo[q] = zo[q] + x0[q];
        }
        SpinorIO<P>::store(x, g.V, se, z);
        SpinorIO<P>::store(x, g.V, so, zo);
    }
}

// ------------------------------------------------------------ SAP half sweep, staged operator
// Same algorithm as sap_half_kernel, but the domain's own forward links and
// clover are copied to shared memory once, so the nmr minimal-residual steps
// read the operator only from shared memory; the block reduction uses one
// barrier per step (double-buffered partials).  FP32 and FP16 storage.
template <class P> struct Staged;
template <> struct Staged<P32> {
    using LC = float4;   // link chunk: 3 per link
    using CC = float4;   // clover chunk: 18 per site
    static constexpr int kLinkChunks = 3, kCloverChunks = 18;
    DEV static void link(const LC* sl, int vbp, int mu, int l, cx<float> u[3][3]) {
        const LC* p = sl + (size_t)mu * 3 * vbp;
        float4 a = p[l], b = p[vbp + l], c = p[2 * vbp + l];
        u[0][0] = {a.x, a.y};
        u[0][1] = {a.z, a.w};
        u[0][2] = {b.x, b.y};
        u[1][0] = {b.z, b.w};
        u[1][1] = {c.x, c.y};
        u[1][2] = {c.z, c.w};
        reconstruct_row2(u);
    }
    DEV static void clover_block(const CC* sc, int vbp, int l, int b, float pr[36]) {
        const CC* p = sc + (size_t)9 * b * vbp;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            float4 t = p[q * vbp + l];
            pr[4 * q] = t.x;
            pr[4 * q + 1] = t.y;
            pr[4 * q + 2] = t.z;
            pr[4 * q + 3] = t.w;
        }
    }
};
template <> struct Staged<P16> {
    using LC = uint2;   // 3 per link
    using CC = uint4;   // 9 per site
    static constexpr int kLinkChunks = 3, kCloverChunks = 9;
    DEV static void link(const LC* sl, int vbp, int mu, int l, cx<float> u[3][3]) {
        const LC* p = sl + (size_t)mu * 3 * vbp;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            uint2 t = p[q * vbp + l];
            const __half2* h = reinterpret_cast<const __half2*>(&t);
            float2 f0 = __half22float2(h[0]), f1 = __half22float2(h[1]);
            int k0 = 2 * q, k1 = 2 * q + 1;
            u[k0 / 3][k0 % 3] = {f0.x, f0.y};
            u[k1 / 3][k1 % 3] = {f1.x, f1.y};
        }
        reconstruct_row2(u);
    }
    DEV static void clover_block(const CC* sc, int vbp, int l, int b, float pr[36]) {
#pragma unroll
        for (int k = 0; k < 36; k += 2) {
            int hidx = 36 * b + k;
            uint4 t = sc[(hidx / 8) * vbp + l];
            const __half2* h = reinterpret_cast<const __half2*>(&t);
            float2 f = __half22float2(h[(hidx % 8) / 2]);
            pr[k] = f.x;
            pr[k + 1] = f.y;
        }
    }
};

// NR right-hand sides per CTA (NR = 2 for batches): thread (slot, l) works on site l of the
// domain for right-hand side NR * (pair index) + slot; the domain's operator is staged once
// and shared by the slots, each slot has its own residual tile and block reduction.
// PS: the storage the operator is staged from (US, UC: its link and clover fields); P32 vectors
// with PS = P16 stage the FP16 copy of the operator (half the shared memory: two CTAs per SM)
// while the residual b - D x still uses the FP32 operator U, C.
template <class P, int NR, class PS = P>
__global__ void __launch_bounds__(256 * NR, (PS::id == 2 && NR == 1) ? 2 : 1)
    sap_half_staged_kernel(Geom g, Blocking bk, int colour, int nmr, int x_mode, const void* __restrict__ U,
                           const void* __restrict__ C, const void* __restrict__ b, void* x, float kappa,
                           int rhs_fast, int nrhs, const void* __restrict__ US, const void* __restrict__ CS) {
    using S = Staged<PS>;
    using LC = typename S::LC;
    using CC = typename S::CC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int vbp = blockDim.x / NR;
    const int slot = threadIdx.x / vbp;
    LC* sl = reinterpret_cast<LC*>(smem_raw);                                     // [4*3][vbp]
    CC* sc = reinterpret_cast<CC*>(sl + (size_t)4 * S::kLinkChunks * vbp);        // [kCloverChunks][vbp]
    cx<float>* rsh = reinterpret_cast<cx<float>*>(sc + (size_t)S::kCloverChunks * vbp) + (size_t)slot * 12 * vbp;
    float* red = reinterpret_cast<float*>(reinterpret_cast<cx<float>*>(sc + (size_t)S::kCloverChunks * vbp) +
                                          (size_t)NR * 12 * vbp) + slot * 192;   // [NR][2][3][32]

    const int k = rhs_fast ? blockIdx.y : blockIdx.x;
    const int rr = NR * (rhs_fast ? blockIdx.x : blockIdx.y) + slot;
    const bool rhs_ok = rr < nrhs;
    const int h0 = bk.C[0] / 2;
    int rest = k / h0;
    int X1 = rest % bk.C[1];
    rest /= bk.C[1];
    int X2 = rest % bk.C[2];
    int X3 = rest / bk.C[2];
    int X0 = 2 * (k % h0) + ((X1 + X2 + X3 + colour) & 1);
    const int Xi = X0 + bk.C[0] * (X1 + bk.C[1] * (X2 + bk.C[2] * X3));

    const int l = threadIdx.x - slot * vbp, lane = l & 31, warp = l >> 5, nw = (vbp + 31) >> 5;
    const bool site = l < bk.Vb;
    const bool active = site && rhs_ok;
    int c[4] = {0, 0, 0, 0}, lc[4] = {0, 0, 0, 0}, s = 0;
    const int lstr[4] = {1, bk.b[0], bk.b[0] * bk.b[1], bk.b[0] * bk.b[1] * bk.b[2]};
    cx<float> r[12], z[12], Ar[12];
    b = (const char*)b + (rhs_ok ? rr : 0) * spinor_bytes<P>(g.V);
    x = (char*)x + (rhs_ok ? rr : 0) * spinor_bytes<P>(g.V);
    if (site) {
        s = block_site(g, bk, Xi, l, c);
        for (int mu = 0; mu < 4; ++mu) lc[mu] = c[mu] % bk.b[mu];
        // stage this site's forward links (slot 0) and clover (the last slot)
        if (slot == 0) {
            const LC* gl = (const LC*)US;
#pragma unroll
            for (int mu = 0; mu < 4; ++mu)
#pragma unroll
                for (int q = 0; q < S::kLinkChunks; ++q)
                    sl[(mu * S::kLinkChunks + q) * vbp + l] =
                        __ldg(gl + ((size_t)mu * S::kLinkChunks + q) * g.V + s);
        }
        if (slot == NR - 1) {
            const CC* gc = (const CC*)CS;
#pragma unroll
            for (int q = 0; q < S::kCloverChunks; ++q) sc[q * vbp + l] = __ldg(gc + (size_t)q * g.V + s);
        }
    }
    if (active) {
        // r = b - D x at this site (global operator; hops may leave the domain)
        SpinorIO<P>::load(b, g.V, s, r);
        if (x_mode != 1) {
            cx<float> psi[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) Ar[q] = czero<float>();
            if (x_mode == 0) {
                SpinorIO<P>::load(x, g.V, s, psi);
                clover_apply<P>(C, g.V, s, psi, Ar);
            }
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                float ph;
                cx<float> u[3][3];
                if (x_mode == 0 || lc[mu] == bk.b[mu] - 1) {
                    int n = neighbour(g, s, c, mu, +1, ph);
                    SpinorIO<P>::load(x, g.V, n, psi);
                    GaugeIO<P>::load(U, g.V, mu, s, u);
                    hop_accum<float>(Ar, psi, u, mu, +1, -kappa * ph);
                }
                if (x_mode == 0 || lc[mu] == 0) {
                    int n = neighbour(g, s, c, mu, -1, ph);
                    SpinorIO<P>::load(x, g.V, n, psi);
                    GaugeIO<P>::load(U, g.V, mu, n, u);
                    hop_accum<float>(Ar, psi, u, mu, -1, -kappa * ph);
                }
            }
#pragma unroll
            for (int q = 0; q < 12; ++q) r[q] = r[q] - Ar[q];
        }
#pragma unroll
        for (int q = 0; q < 12; ++q) z[q] = czero<float>();
        DomainVec<float>::put(rsh, vbp, l, r);
    }
    for (int it = 0; it < nmr; ++it) {
        __syncthreads();   // r (and, first time, the staged operator) visible
        float part[3] = {0.f, 0.f, 0.f};
        if (active) {
            float pr[36];
            S::clover_block(sc, vbp, l, 0, pr);
            clover_block_apply<float>(pr, r, Ar);
            S::clover_block(sc, vbp, l, 1, pr);
            clover_block_apply<float>(pr, r + 6, Ar + 6);
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                cx<float> u[3][3], psi[12];
                if (lc[mu] != bk.b[mu] - 1) {
                    DomainVec<float>::get(rsh, vbp, l + lstr[mu], psi);
                    S::link(sl, vbp, mu, l, u);
                    hop_accum<float>(Ar, psi, u, mu, +1, -kappa);
                }
                if (lc[mu] != 0) {
                    DomainVec<float>::get(rsh, vbp, l - lstr[mu], psi);
                    S::link(sl, vbp, mu, l - lstr[mu], u);
                    hop_accum<float>(Ar, psi, u, mu, -1, -kappa);
                }
            }
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                // <Ar, r> and |Ar|^2 as fused multiply-adds
                part[0] = fma(Ar[q].re, r[q].re, part[0]);
                part[0] = fma(Ar[q].im, r[q].im, part[0]);
                part[1] = fma(Ar[q].re, r[q].im, part[1]);
                part[1] = fma(-Ar[q].im, r[q].re, part[1]);
                part[2] = fma(Ar[q].re, Ar[q].re, part[2]);
                part[2] = fma(Ar[q].im, Ar[q].im, part[2]);
            }
        }
        // one-barrier block reduction into buffer (it & 1)
        float* rb = red + (it & 1) * 96;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float v = warp_sum(part[q]);
            if (lane == 0) rb[q * 32 + warp] = v;
        }
        __syncthreads();
        float tot[3] = {0.f, 0.f, 0.f};
        for (int w = 0; w < nw; ++w) {
            tot[0] += rb[w];
            tot[1] += rb[32 + w];
            tot[2] += rb[64 + w];
        }
        cx<float> alpha = czero<float>();
        if (tot[2] > 0.f) alpha = {tot[0] / tot[2], tot[1] / tot[2]};
        if (active) {
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                cfma(z[q], alpha, r[q]);
                cfma(r[q], -alpha, Ar[q]);
            }
            DomainVec<float>::put(rsh, vbp, l, r);
        }
    }
    if (active) {
        if (x_mode == 0) {
            cx<float> x0[12];
            SpinorIO<P>::load(x, g.V, s, x0);
#pragma unroll
            for (int q = 0; q < 12; ++q) z[q] = z[q] + x0[q];
        }
        SpinorIO<P>::store(x, g.V, s, z);
    }
}

template <class P>
size_t sap_staged_smem(int vbp, int nr = 1) {
    using S = Staged<P>;
    return (size_t)vbp * (4 * S::kLinkChunks * sizeof(typename S::LC) + S::kCloverChunks * sizeof(typename S::CC) +
                          nr * 12 * sizeof(cx<float>)) +
           nr * 2 * 96 * sizeof(float);
}

template <class P, class PS = P>
cudaError_t sap_half_staged_impl(const GeomH& gh, const BlockH& bh, int colour, int nmr, int x_mode, const void* U,
                                 const void* C, const void* b, void* x, double kappa, int nrhs, cudaStream_t st,
                                 const void* US = nullptr, const void* CS = nullptr) {
    if (!US) US = U;
    if (!CS) CS = C;
    Geom g = make_geom(gh);
    Blocking bk = make_blocking(gh, bh);
    int threads = (bk.Vb + 31) / 32 * 32;
    if (threads > 256) return cudaErrorInvalidValue;
    const int ndom = bk.Vc / 2;
    // batches: two right-hand sides per CTA share the staged operator
    const int nr = nrhs > 1 ? 2 : 1;
    const int npair = (nrhs + nr - 1) / nr;
    const int fast = npair > 1 && ndom <= 65535;
    const dim3 grid = fast ? dim3(npair, ndom) : dim3(ndom, npair);
    size_t smem = sap_staged_smem<PS>(threads, nr);
    auto fn = nr == 2 ? sap_half_staged_kernel<P, 2, PS> : sap_half_staged_kernel<P, 1, PS>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    (note_launch(), fn<<<grid, threads * nr, smem, st>>>(g, bk, colour, nmr, x_mode, U, C, b, x, (float)kappa, fast,
                                                          nrhs, US, CS));
    return cudaGetLastError();
}

template <class P>
cudaError_t sap_half_impl(const GeomH& gh, const BlockH& bh, int colour, int nmr, int x_mode, const void* U,
                          const void* C, const void* b, void* x, double kappa, int nrhs, cudaStream_t st,
                          bool pair = false) {
    Geom g = make_geom(gh);
    Blocking bk = make_blocking(gh, bh);
    int threads = (bk.Vb + 31) / 32 * 32;
    if (threads > 512) return cudaErrorInvalidValue;
    // two right-hand sides per CTA (variant 2, batches, FP32/FP16, blocks of <= 256 sites)
    const int nr = (pair && nrhs > 1 && threads <= 256 && P::id != 0) ? 2 : 1;
    size_t smem = (size_t)nr * 12 * threads * sizeof(cx<typename P::T>) + nr * 2 * 3 * 32 * sizeof(typename P::T);
    int ndom = bk.Vc / 2;
    const int ngrp = (nrhs + nr - 1) / nr;
    // right-hand side as the fast grid index when the domains fit the y dimension
    const int fast = ngrp > 1 && ndom <= 65535;
    const dim3 grid = fast ? dim3(ngrp, ndom) : dim3(ndom, ngrp);
    const typename P::T kp = (typename P::T)kappa;
    if constexpr (P::id != 0) {
        if (nr == 2) {
            auto fn = sap_half_kernel<P, 256, 2>;
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            (note_launch(), fn<<<grid, 2 * threads, smem, st>>>(g, bk, colour, nmr, x_mode, U, C, b, x, kp, fast,
                                                                 nrhs));
            return cudaGetLastError();
        }
    }
    if (threads <= 256) {
        auto fn = sap_half_kernel<P, 256, 1>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        (note_launch(), fn<<<grid, threads, smem, st>>>(g, bk, colour, nmr, x_mode, U, C, b, x, kp, fast, nrhs));
    } else {
        auto fn = sap_half_kernel<P, 512, 1>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        (note_launch(), fn<<<grid, threads, smem, st>>>(g, bk, colour, nmr, x_mode, U, C, b, x, kp, fast, nrhs));
    }
    return cudaGetLastError();
}

// launch shape of the stencil per precision, chosen by the autotuner (dirac_set_shape):
// threads per CTA and the grid cap in CTAs per SM (grid-stride loop beyond it)
struct DiracShape {
    int threads, per_sm, mb;   // mb: register budget as resident CTAs per SM (0 = the default)
};
DiracShape g_dirac_shape[3] = {{kThreads, 16, 0}, {kThreads, 16, 0}, {kThreads, 16, 0}};

template <class P>
cudaError_t dirac_impl(const GeomH& gh, const BlockH* sb, const void* U, const void* C, const void* in, void* out,
                       const void* b, double kappa, int nrhs, cudaStream_t st) {
    Geom g = make_geom(gh);
    Blocking bk;
    BlockH one = {{1, 1, 1, 1}};
    bk = make_blocking(gh, sb ? *sb : one);
    const DiracShape sh = g_dirac_shape[P::id];
    int blocks = (g.V + sh.threads - 1) / sh.threads;
    const int cap = device_sms() * sh.per_sm;
    if (blocks > cap) blocks = cap;
    dim3 grid(blocks, nrhs);
    const int th = sh.threads;
    using T = typename P::T;
    if (sb) {
        if (b) (note_launch(), dirac_kernel<P, true, true><<<grid, th, 0, st>>>(g, bk, U, C, in, out, b, (T)kappa));
        else (note_launch(), dirac_kernel<P, true, false><<<grid, th, 0, st>>>(g, bk, U, C, in, out, b, (T)kappa));
        return cudaGetLastError();
    }
    if constexpr (P::id != 0) {
        if (sh.mb == 2) {
            if (b) (note_launch(), dirac_kernel<P, false, true, 2><<<grid, th, 0, st>>>(g, bk, U, C, in, out, b, (T)kappa));
            else (note_launch(), dirac_kernel<P, false, false, 2><<<grid, th, 0, st>>>(g, bk, U, C, in, out, b, (T)kappa));
            return cudaGetLastError();
        }
    }
    if (b) (note_launch(), dirac_kernel<P, false, true><<<grid, th, 0, st>>>(g, bk, U, C, in, out, b, (T)kappa));
    else (note_launch(), dirac_kernel<P, false, false><<<grid, th, 0, st>>>(g, bk, U, C, in, out, b, (T)kappa));
    return cudaGetLastError();
}

// sigma_munu = [gamma_mu, gamma_nu] / (2i) in the chiral basis, chirality blocks.
// gamma_mu = [[0, e_mu], [e_mu^dag, 0]] so gamma_mu gamma_nu = diag(e_mu e_nu^dag, e_mu^dag e_nu).
struct C2 {
    double re, im;
};
static C2 cm(C2 a, C2 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
static void e_matrix(int mu, C2 e[2][2], bool dag) {
    C2 z = {0, 0}, one = {1, 0}, I = {0, 1}, mI = {0, -1}, mone = {-1, 0};
    C2 m[2][2];
    switch (mu) {
        case 0: m[0][0] = z; m[0][1] = I; m[1][0] = I; m[1][1] = z; break;
        case 1: m[0][0] = z; m[0][1] = one; m[1][0] = mone; m[1][1] = z; break;
        case 2: m[0][0] = I; m[0][1] = z; m[1][0] = z; m[1][1] = mI; break;
        default: m[0][0] = one; m[0][1] = z; m[1][0] = z; m[1][1] = one; break;
    }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) e[i][j] = dag ? C2{m[j][i].re, -m[j][i].im} : m[i][j];
}
static void mm2(C2 a[2][2], C2 b[2][2], C2 c[2][2]) {
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            C2 t1 = cm(a[i][0], b[0][j]), t2 = cm(a[i][1], b[1][j]);
            c[i][j] = {t1.re + t2.re, t1.im + t2.im};
        }
}
static bool sigma_uploaded = false;
static cudaError_t upload_sigma() {
    if (sigma_uploaded) return cudaSuccess;
    double2 h[6][2][2][2];
    int plane = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
            C2 em[2][2], emd[2][2], en[2][2], endg[2][2];
            e_matrix(mu, em, false);
            e_matrix(mu, emd, true);
            e_matrix(nu, en, false);
            e_matrix(nu, endg, true);
            C2 p[2][2][2], q[2][2][2];
            mm2(em, endg, p[0]);   // upper block of gamma_mu gamma_nu
            mm2(emd, en, p[1]);    // lower block
            mm2(en, emd, q[0]);
            mm2(endg, em, q[1]);
            for (int b = 0; b < 2; ++b)
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) {
                        C2 d = {p[b][i][j].re - q[b][i][j].re, p[b][i][j].im - q[b][i][j].im};
                        // d / (2i) = -i d / 2
                        h[plane][b][i][j] = make_double2(d.im / 2.0, -d.re / 2.0);
                    }
        }
    cudaError_t e = cudaMemcpyToSymbol(c_sigma, h, sizeof(h));
    if (e == cudaSuccess) sigma_uploaded = true;
    return e;
}

}  // namespace

// ============================================================ launchers
size_t fine_spinor_bytes(int prec, int V) {
    return prec == 0 ? spinor_bytes<P64>(V) : prec == 1 ? spinor_bytes<P32>(V) : spinor_bytes<P16>(V);
}
size_t fine_gauge_bytes(int prec, int V) {
    size_t per = prec == 0 ? GaugeIO<P64>::bytes_per_link : prec == 1 ? GaugeIO<P32>::bytes_per_link
                                                       : prec == 3 ? GaugeIO<PDD>::bytes_per_link
                                                                   : GaugeIO<P16>::bytes_per_link;
    return 4 * per * (size_t)V;
}
size_t fine_clover_bytes(int prec, int V) {
    size_t per = prec == 0 ? CloverIO<P64>::bytes_per_site : prec == 1 ? CloverIO<P32>::bytes_per_site
                                                        : prec == 3 ? CloverIO<PDD>::bytes_per_site
                                                                    : CloverIO<P16>::bytes_per_site;
    return per * (size_t)V;
}

cudaError_t launch_pack_spinor(int prec, const GeomH& gh, const void* canon, void* internal, int nrhs,
                               cudaStream_t st) {
    Geom g = make_geom(gh);
    dim3 grid(grid_for(g.V, kThreads), nrhs);
    if (((uintptr_t)canon & 15) == 0) {
        const dim3 gt(grid_for(g.V, kTile), nrhs);
        if (prec == 0) (note_launch(), pack_tiled_kernel<P64, double><<<gt, kTile, 0, st>>>(g, (const double*)canon, internal));
        else if (prec == 1) (note_launch(), pack_tiled_kernel<P32, float><<<gt, kTile, 0, st>>>(g, (const float*)canon, internal));
        else (note_launch(), pack_tiled_kernel<P16, float><<<gt, kTile, 0, st>>>(g, (const float*)canon, internal));
        return cudaGetLastError();
    }
    if (prec == 0) (note_launch(), pack_kernel<P64, double><<<grid, kThreads, 0, st>>>(g, (const double*)canon, internal, nrhs));
    else if (prec == 1) (note_launch(), pack_kernel<P32, float><<<grid, kThreads, 0, st>>>(g, (const float*)canon, internal, nrhs));
    else (note_launch(), pack_kernel<P16, float><<<grid, kThreads, 0, st>>>(g, (const float*)canon, internal, nrhs));
    return cudaGetLastError();
}
cudaError_t launch_unpack_spinor(int prec, const GeomH& gh, const void* internal, void* canon, int nrhs,
                                 cudaStream_t st) {
    Geom g = make_geom(gh);
    dim3 grid(grid_for(g.V, kThreads), nrhs);
    if (((uintptr_t)canon & 15) == 0) {
        const dim3 gt(grid_for(g.V, kTile), nrhs);
        if (prec == 0) (note_launch(), unpack_tiled_kernel<P64, double><<<gt, kTile, 0, st>>>(g, internal, (double*)canon));
        else if (prec == 1) (note_launch(), unpack_tiled_kernel<P32, float><<<gt, kTile, 0, st>>>(g, internal, (float*)canon));
        else (note_launch(), unpack_tiled_kernel<P16, float><<<gt, kTile, 0, st>>>(g, internal, (float*)canon));
        return cudaGetLastError();
    }
    if (prec == 0) (note_launch(), unpack_kernel<P64, double><<<grid, kThreads, 0, st>>>(g, internal, (double*)canon, nrhs));
    else if (prec == 1) (note_launch(), unpack_kernel<P32, float><<<grid, kThreads, 0, st>>>(g, internal, (float*)canon, nrhs));
    else (note_launch(), unpack_kernel<P16, float><<<grid, kThreads, 0, st>>>(g, internal, (float*)canon, nrhs));
    return cudaGetLastError();
}
cudaError_t launch_convert_spinor(int pi, int po, const GeomH& gh, const void* in, void* out, int nrhs,
                                  cudaStream_t st) {
    Geom g = make_geom(gh);
    dim3 grid(grid_for(g.V, kThreads), nrhs);
#define CONV(A, B) (note_launch(), convert_kernel<A, B><<<grid, kThreads, 0, st>>>(g, in, out))
    if (pi == 0 && po == 1) CONV(P64, P32);
    else if (pi == 1 && po == 0) CONV(P32, P64);
    else if (pi == 0 && po == 2) CONV(P64, P16);
    else if (pi == 2 && po == 0) CONV(P16, P64);
    else if (pi == 1 && po == 2) CONV(P32, P16);
    else if (pi == 2 && po == 1) CONV(P16, P32);
    else if (pi == 0 && po == 0) CONV(P64, P64);
    else if (pi == 1 && po == 1) CONV(P32, P32);
    else CONV(P16, P16);
#undef CONV
    return cudaGetLastError();
}
cudaError_t launch_gauge_convert(int prec, const GeomH& gh, const double* canon, void* internal, cudaStream_t st) {
    Geom g = make_geom(gh);
    (note_launch(), gauge_convert_kernel<<<grid_for(g.V, kThreads), kThreads, 0, st>>>(g, canon, internal, prec));
    return cudaGetLastError();
}
cudaError_t launch_clover_build(int prec, const GeomH& gh, const void* U64, double kappa, double csw, void* clover,
                                cudaStream_t st) {
    cudaError_t e = upload_sigma();
    if (e != cudaSuccess) return e;
    Geom g = make_geom(gh);
    int grid = grid_for(g.V, 128);
    if (prec == 0) (note_launch(), clover_build_kernel<P64><<<grid, 128, 0, st>>>(g, U64, kappa, csw, clover));
    else if (prec == 1) (note_launch(), clover_build_kernel<P32><<<grid, 128, 0, st>>>(g, U64, kappa, csw, clover));
    else if (prec == 3) (note_launch(), clover_build_kernel<PDD><<<grid, 128, 0, st>>>(g, U64, kappa, csw, clover));
    else (note_launch(), clover_build_kernel<P16><<<grid, 128, 0, st>>>(g, U64, kappa, csw, clover));
    return cudaGetLastError();
}
cudaError_t launch_clover_expand(const GeomH& gh, const void* C64, double* out, cudaStream_t st) {
    Geom g = make_geom(gh);
    (note_launch(), clover_expand_kernel<<<grid_for(g.V, kThreads), kThreads, 0, st>>>(g, C64, out));
    return cudaGetLastError();
}
void dirac_set_shape(int prec, int threads, int per_sm, int mb) {
    if (prec < 0 || prec > 2 || threads < 32 || threads > kThreads || threads % 32 || per_sm < 1) return;
    if (mb != 0 && mb != 2 && mb != 3) return;
    g_dirac_shape[prec] = {threads, per_sm, prec == 0 ? 0 : mb};
}
void dirac_get_shape(int prec, int* threads, int* per_sm, int* mb) {
    *threads = g_dirac_shape[prec].threads;
    *per_sm = g_dirac_shape[prec].per_sm;
    if (mb) *mb = g_dirac_shape[prec].mb;
}
cudaError_t launch_dirac(int prec, const GeomH& g, const BlockH* sb, const void* U, const void* C, const void* in,
                         void* out, const void* b, double kappa, int nrhs, cudaStream_t st) {
    if (prec == 0) return dirac_impl<P64>(g, sb, U, C, in, out, b, kappa, nrhs, st);
    if (prec == 1) return dirac_impl<P32>(g, sb, U, C, in, out, b, kappa, nrhs, st);
    return dirac_impl<P16>(g, sb, U, C, in, out, b, kappa, nrhs, st);
}
cudaError_t launch_dirac_mixed(const GeomH& gh, const void* Udd, const void* Cdd, const void* in32, void* out64,
                               double kappa, int nrhs, cudaStream_t st) {
    Geom g = make_geom(gh);
    dim3 grid(grid_for(g.V, kThreads), nrhs);
    (note_launch(), dirac_mixed_kernel<<<grid, kThreads, 0, st>>>(g, Udd, Cdd, in32, out64, split_double(kappa)));
    return cudaGetLastError();
}
cudaError_t launch_spinor_axpy_mixed(const GeomH& gh, int k, const double2* c, const void* const* z, void* x,
                                     cudaStream_t st, bool pair) {
    if (k < 1 || k > 20) return cudaErrorInvalidValue;
    ZList zl;
    for (int j = 0; j < k; ++j) {
        zl.p[j] = z[j];
        zl.c[j] = c[j];
    }
    Geom g = make_geom(gh);
    if (pair) (note_launch(), spinor_axpy_mixed_df_kernel<<<grid_for(g.V, kThreads), kThreads, 0, st>>>(g, k, zl, x));
    else (note_launch(), spinor_axpy_mixed_kernel<<<grid_for(g.V, kThreads), kThreads, 0, st>>>(g, k, zl, x));
    return cudaGetLastError();
}
template <class P>
cudaError_t sap_half_eo_impl(const GeomH& gh, const BlockH& bh, int colour, int nmr, int x_mode, const void* U,
                             const void* C, const void* Ci, const void* b, void* x, double kappa, int nrhs,
                             cudaStream_t st) {
    Geom g = make_geom(gh);
    Blocking bk = make_blocking(gh, bh);
    if (bk.b[0] % 2 != 0) return cudaErrorInvalidValue;   // pairs of x-neighbours of opposite parity
    const int threads = ((bk.Vb / 2) + 31) / 32 * 32;
    if (threads > 256) return cudaErrorInvalidValue;
    using T = typename P::T;
    const size_t smem = (size_t)12 * (2 * threads) * sizeof(cx<T>) + (size_t)12 * threads * sizeof(cx<T>) +
                        3 * 32 * sizeof(T);
    const int ndom = bk.Vc / 2;
    const int fast = nrhs > 1 && ndom <= 65535;
    const dim3 grid = fast ? dim3(nrhs, ndom) : dim3(ndom, nrhs);
    cudaError_t e = cudaFuncSetAttribute(sap_half_eo_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    (note_launch(), sap_half_eo_kernel<P><<<grid, threads, smem, st>>>(g, bk, colour, nmr, x_mode, U, C, Ci, b, x,
                                                                      (T)kappa, fast));
    return cudaGetLastError();
}

cudaError_t launch_sap_half_eo(int prec, const GeomH& g, const BlockH& bk, int colour, int nmr, int x_mode,
                               const void* U, const void* C, const void* Ci, const void* b, void* x, double kappa,
                               int nrhs, cudaStream_t st) {
    if (prec == 0) return sap_half_eo_impl<P64>(g, bk, colour, nmr, x_mode, U, C, Ci, b, x, kappa, nrhs, st);
    if (prec == 1) return sap_half_eo_impl<P32>(g, bk, colour, nmr, x_mode, U, C, Ci, b, x, kappa, nrhs, st);
    return sap_half_eo_impl<P16>(g, bk, colour, nmr, x_mode, U, C, Ci, b, x, kappa, nrhs, st);
}
bool sap_eo_supported(const BlockH& bk) {
    const int vb = bk.b[0] * bk.b[1] * bk.b[2] * bk.b[3];
    return bk.b[0] % 2 == 0 && vb <= 512;
}
cudaError_t launch_clover_invert(int prec, const GeomH& gh, const void* C64, void* out, cudaStream_t st) {
    Geom g = make_geom(gh);
    int grid = grid_for(g.V, 128);
    if (prec == 0) (note_launch(), clover_invert_kernel<P64><<<grid, 128, 0, st>>>(g, C64, out));
    else if (prec == 1) (note_launch(), clover_invert_kernel<P32><<<grid, 128, 0, st>>>(g, C64, out));
    else (note_launch(), clover_invert_kernel<P16><<<grid, 128, 0, st>>>(g, C64, out));
    return cudaGetLastError();
}

cudaError_t launch_sap_half_variant(int variant, int prec, const GeomH& g, const BlockH& bk, int colour, int nmr,
                                    int x_mode, const void* U, const void* C, const void* b, void* x, double kappa,
                                    int nrhs, cudaStream_t st) {
    if (variant == 1 && prec == 1)
        return sap_half_staged_impl<P32>(g, bk, colour, nmr, x_mode, U, C, b, x, kappa, nrhs, st);
    if (variant == 1 && prec == 2)
        return sap_half_staged_impl<P16>(g, bk, colour, nmr, x_mode, U, C, b, x, kappa, nrhs, st);
    const bool pair = variant == 2;
    if (prec == 0) return sap_half_impl<P64>(g, bk, colour, nmr, x_mode, U, C, b, x, kappa, nrhs, st, pair);
    if (prec == 1) return sap_half_impl<P32>(g, bk, colour, nmr, x_mode, U, C, b, x, kappa, nrhs, st, pair);
    return sap_half_impl<P16>(g, bk, colour, nmr, x_mode, U, C, b, x, kappa, nrhs, st, pair);
}
cudaError_t launch_sap_half_staged16(const GeomH& g, const BlockH& bk, int colour, int nmr, int x_mode,
                                     const void* U32, const void* C32, const void* U16, const void* C16,
                                     const void* b, void* x, double kappa, int nrhs, cudaStream_t st) {
    return sap_half_staged_impl<P32, P16>(g, bk, colour, nmr, x_mode, U32, C32, b, x, kappa, nrhs, st, U16, C16);
}
bool sap_staged_supported(int prec, const BlockH& bk) {
    int vb = bk.b[0] * bk.b[1] * bk.b[2] * bk.b[3];
    return (prec == 1 || prec == 2) && vb <= 256;
}
cudaError_t launch_sap_half(int prec, const GeomH& g, const BlockH& bk, int colour, int nmr, int x_mode, const void* U,
                            const void* C, const void* b, void* x, double kappa, cudaStream_t st) {
    if (prec == 0) return sap_half_impl<P64>(g, bk, colour, nmr, x_mode, U, C, b, x, kappa, 1, st);
    if (prec == 1) return sap_half_impl<P32>(g, bk, colour, nmr, x_mode, U, C, b, x, kappa, 1, st);
    return sap_half_impl<P16>(g, bk, colour, nmr, x_mode, U, C, b, x, kappa, 1, st);
}

// ---------------------------------------------------------------- ragged batches
size_t ragged_dev_bytes() { return sizeof(RaggedDev); }

int ragged_dev_fill(void* dst, const RaggedProbH& h) {
    if (h.nbasis < 1 || h.nbasis > kRaggedMaxBasis) return -1;
    RaggedDev q = {};
    q.g = make_geom(h.g);
    q.bk = make_blocking(h.g, h.blk);
    q.nvec = h.nvec;
    q.kappa = h.kappa;
    q.kappa32 = (float)h.kappa;
    q.U32 = h.U32;
    q.C32 = h.C32;
    q.Udd = h.Udd;
    q.Cdd = h.Cdd;
    q.vecs = h.vecs;
    q.v = h.v;
    q.f32 = h.f32;
    q.f32b = h.f32b;
    q.bc = h.bc;
    q.xc = h.xc;
    q.z = h.z;
    q.w = h.w;
    for (int i = 0; i < h.nbasis; ++i) q.basis[i] = h.basis[i];
    q.vnext = h.vnext;
    q.gs_part = h.gs_part;
    q.gs_coef = h.gs_coef;
    q.n = h.n;
    q.R = h.R;
    q.U64 = h.U64;
    q.C64 = h.C64;
    q.b64 = h.b64;
    q.x64 = h.x64;
    q.r64 = h.r64;
    q.rsrc = h.rsrc;
    q.npart = h.npart;
    q.nval = h.nval;
    if (h.k < 0 || h.k > kRaggedMaxBasis) return -1;
    q.k = h.k;
    for (int i = 0; i < h.k; ++i) {
        q.zb[i] = h.zb[i];
        q.yc[i] = h.yc[i];
    }
    q.canon_in = h.canon_in;
    q.canon_out = h.canon_out;
    if (h.sap_nr != 1 && h.sap_nr != 2) return -1;
    q.sap_nr = h.sap_nr;
    memcpy(dst, &q, sizeof q);
    return 0;
}

int ragged_site_ctas(int V) {
    int c = (V + kThreads - 1) / kThreads;
    return c < 1 ? 1 : c;
}

cudaError_t launch_convert_ragged(const void* d, const int* off, int np, int ctas, cudaStream_t st) {
    (note_launch(), convert_ragged_kernel<<<ctas, kThreads, 0, st>>>((const RaggedDev*)d, off, np));
    return cudaGetLastError();
}
cudaError_t launch_dirac_mixed_ragged(const void* d, const int* off, int np, int ctas, cudaStream_t st) {
    (note_launch(), dirac_mixed_ragged_kernel<<<ctas, kThreads, 0, st>>>((const RaggedDev*)d, off, np));
    return cudaGetLastError();
}
int ragged_sap_threads(int max_vb) {
    const int t = (max_vb + 31) / 32 * 32;
    return t > 128 ? 256 : 2 * t;
}
int ragged_sap_nr(int vb, int max_vb) {
    const int half = ragged_sap_threads(max_vb) / 2;   // a multiple of 32
    return vb <= half ? 2 : 1;
}
cudaError_t launch_sap_half_ragged(const void* d, const int* off, int np, int ctas, int max_vb, int colour, int nmr,
                                   cudaStream_t st) {
    const int threads = ragged_sap_threads(max_vb);
    if (max_vb > 256 || ctas < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)12 * threads * sizeof(cx<float>) + 2 * 2 * 3 * 32 * sizeof(float);
    (note_launch(), sap_half_ragged_kernel<<<ctas, threads, smem, st>>>((const RaggedDev*)d, off, np, colour, nmr));
    return cudaGetLastError();
}
cudaError_t launch_pack_ragged(const void* d, const int* off, int np, int ctas, cudaStream_t st) {
    (note_launch(), pack_ragged_kernel<<<ctas, kThreads, 0, st>>>((const RaggedDev*)d, off, np));
    return cudaGetLastError();
}
cudaError_t launch_unpack_ragged(const void* d, const int* off, int np, int ctas, cudaStream_t st) {
    (note_launch(), unpack_ragged_kernel<<<ctas, kThreads, 0, st>>>((const RaggedDev*)d, off, np));
    return cudaGetLastError();
}
cudaError_t launch_resid_ragged(const void* d, const int* off, int np, int ctas, bool pair, cudaStream_t st) {
    if (!pair) {
        (note_launch(), resid64_ragged_kernel<<<ctas, kThreads, 0, st>>>((const RaggedDev*)d, off, np));
        return cudaGetLastError();
    }
    (note_launch(), split_ragged_kernel<<<ctas, kThreads, 0, st>>>((const RaggedDev*)d, off, np));
    (note_launch(), resid_ragged_kernel<<<ctas, kThreads, 0, st>>>((const RaggedDev*)d, off, np));
    return cudaGetLastError();
}
cudaError_t launch_xupdate_ragged(const void* d, const int* off, int np, int ctas, cudaStream_t st) {
    (note_launch(), xupdate_ragged_kernel<<<ctas, kThreads, 0, st>>>((const RaggedDev*)d, off, np));
    return cudaGetLastError();
}
cudaError_t launch_dirac_dd(const GeomH& gh, const void* Udd, const void* Cdd, const void* U32, const void* C32,
                            const void* in64, void* out64, const void* b64, double kappa, int nrhs, void* hi,
                            void* lo, cudaStream_t st) {
    Geom g = make_geom(gh);
    dim3 grid(grid_for(g.V, kThreads), nrhs);
    (note_launch(), split_kernel<<<grid, kThreads, 0, st>>>(g, in64, hi, lo));
    if (b64)
        (note_launch(), dirac_hilo_kernel<true><<<grid, kThreads, 0, st>>>(g, Udd, Cdd, U32, C32, hi, lo, out64, b64,
                                                                            split_double(kappa), (float)kappa));
    else
        (note_launch(), dirac_hilo_kernel<false><<<grid, kThreads, 0, st>>>(g, Udd, Cdd, U32, C32, hi, lo, out64,
                                                                             nullptr, split_double(kappa),
                                                                             (float)kappa));
    return cudaGetLastError();
}
