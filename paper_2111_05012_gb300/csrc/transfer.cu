// Transfer between the fine lattice and the first coarse lattice (Sec. 3):
// restriction x(I) = <I|x> (Eq. 5), prolongation |x'> = sum_I x(I)|I> (Eq. 6),
// the block orthonormalisation <I|J> = delta_IJ and the Galerkin coarse
// operator D_c(I, J) = <I|D|J> (Eq. 7).  |X, s, i> is test vector i projected
// to chirality s (spins 0,1 or 2,3) and restricted to block X; coarse dof
// index I = s * nvec + i.  One CTA works on one block, one thread per site.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace {

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

template <typename TC> struct CStore;
template <> struct CStore<double> {
    DEV static void st(void* p, size_t i, cx<double> v) { ((double2*)p)[i] = make_double2(v.re, v.im); }
    DEV static cx<double> ld(const void* p, size_t i) {
        double2 t = ((const double2*)p)[i];
        return {t.x, t.y};
    }
};
template <> struct CStore<float> {
    DEV static void st(void* p, size_t i, cx<float> v) { ((float2*)p)[i] = make_float2(v.re, v.im); }
    DEV static cx<float> ld(const void* p, size_t i) {
        float2 t = ((const float2*)p)[i];
        return {t.x, t.y};
    }
};

// ------------------------------------------------------------ raw vector loads
// A test vector at one site as loaded from memory, unpacked only when used, so
// that the loads of several vectors can be in flight together without holding
// all of them unpacked in registers.
template <class PV> struct RawSite;
template <> struct RawSite<P64> {
    double2 r[12];
    DEV void load(const void* base, int V, int s) {
#pragma unroll
        for (int k = 0; k < 12; ++k) r[k] = __ldg((const double2*)base + (size_t)k * V + s);
    }
    DEV cx<double> get(int k) const { return {r[k].x, r[k].y}; }
};
template <> struct RawSite<P32> {
    float4 r[6];
    DEV void load(const void* base, int V, int s) {
#pragma unroll
        for (int c = 0; c < 6; ++c) r[c] = __ldg((const float4*)base + (size_t)c * V + s);
    }
    DEV cx<float> get(int k) const {
        const float4 t = r[k >> 1];
        return (k & 1) ? cx<float>{t.z, t.w} : cx<float>{t.x, t.y};
    }
};
template <> struct RawSite<P16> {   // three uint4 of halves, then the per-site scale (SpinorIO<P16> layout)
    uint4 r[3];
    float sc;
    DEV void load(const void* base, int V, int s) {
        const uint4* p = (const uint4*)base;
#pragma unroll
        for (int c = 0; c < 3; ++c) r[c] = __ldg(p + (size_t)c * V + s);
        sc = __ldg((const float*)(p + (size_t)3 * V) + s);
    }
    DEV cx<float> get(int k) const {
        const uint4 t = r[k >> 2];
        const unsigned w = (k & 3) == 0 ? t.x : (k & 3) == 1 ? t.y : (k & 3) == 2 ? t.z : t.w;
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w));
        return {f.x * sc, f.y * sc};
    }
};
// vectors whose loads a thread keeps in flight together
template <class PV> constexpr int kVecGroup = PV::id == 2 ? 4 : 2;

// Warp sums of N values per lane (N a power of two, N <= 32) with 2N - 1 + log2(32/N)
// shuffles instead of 5N: each halving step pairs lanes l and l^off, every lane keeping
// one half of its values (the lower half if its bit off is clear) plus the partner's
// copy of that half.  Afterwards lane l holds the total of value sum_t bit(l, 4-t) * N/2^(t+1)
// (see transposed_index), duplicated over the lanes that differ only in the low bits.
template <int N, typename T> DEV T transposed_warp_sum(T (&v)[N], int lane) {
#pragma unroll
    for (int t = 0, h = N / 2, off = 16; h >= 1; ++t, h /= 2, off /= 2) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const T keep = up ? v[k + h] : v[k];
            const T give = up ? v[k] : v[k + h];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, give, off);
        }
    }
    T r = v[0];
#pragma unroll
    for (int off = 16 / N; off >= 1; off /= 2) r += __shfl_xor_sync(0xffffffffu, r, off);
    return r;
}
template <int N> DEV int transposed_index(int lane) {
    int idx = 0;
#pragma unroll
    for (int t = 0, h = N / 2, off = 16; h >= 1; ++t, h /= 2, off /= 2)
        if (lane & off) idx += h;
    return idx;
}

// ------------------------------------------------------------ restriction
// One CTA per block, one thread per site: the site's share of <X,s,i|psi> for a
// group of test vectors (their loads in flight together), summed over the warp
// by transposed shuffles and over the warps in shared memory.
template <class PF, class PV, typename TC>
DEV void restrict_body(const Geom& g, const Blocking& bk, int nvec, const void* __restrict__ vecs,
                       const void* __restrict__ fine, void* coarse, int by, int gy) {
    using T = typename PF::T;
    constexpr int G = kVecGroup<PV>, NQ = 4 * G;   // per vector: d0.re, d0.im, d1.re, d1.im
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* part = reinterpret_cast<cx<T>*>(smem_raw);   // [nwarps][2*nvec]
    T* partf = reinterpret_cast<T*>(smem_raw);
    const int nc = 2 * nvec;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const size_t vb = spinor_bytes<PV>(g.V);
    const int qi = transposed_index<NQ>(lane);
    const bool writer = (lane & (32 / NQ - 1)) == 0;
    for (int Xi = by; Xi < bk.Vc; Xi += gy) {
        const int l = threadIdx.x;
        const bool active = l < bk.Vb;
        int c[4], s = 0;
        cx<T> psi[12];
        if (active) {
            s = block_site(g, bk, Xi, l, c);
            SpinorIO<PF>::load(fine, g.V, s, psi);
        }
        for (int i0 = 0; i0 < nvec; i0 += G) {
            RawSite<PV> raw[G];
            if (active) {
#pragma unroll
                for (int u = 0; u < G; ++u)
                    if (i0 + u < nvec) raw[u].load((const char*)vecs + (size_t)(i0 + u) * vb, g.V, s);
            }
            T q[NQ];
#pragma unroll
            for (int u = 0; u < G; ++u) {
                cx<T> d0 = czero<T>(), d1 = czero<T>();
                if (active && i0 + u < nvec) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        cfmac(d0, ccast<T>(raw[u].get(k)), psi[k]);
                        cfmac(d1, ccast<T>(raw[u].get(6 + k)), psi[6 + k]);
                    }
                }
                q[4 * u] = d0.re;
                q[4 * u + 1] = d0.im;
                q[4 * u + 2] = d1.re;
                q[4 * u + 3] = d1.im;
            }
            const T tot = transposed_warp_sum<NQ>(q, lane);
            const int u = qi >> 2, comp = qi & 3, i = i0 + u;
            if (writer && i < nvec) partf[2 * (warp * nc + (comp < 2 ? i : nvec + i)) + (comp & 1)] = tot;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < nc; j += blockDim.x) {
            cx<T> t = czero<T>();
            for (int w = 0; w < nw; ++w) t = t + part[w * nc + j];
            CStore<TC>::st(coarse, (size_t)Xi * nc + j, ccast<TC>(t));
        }
        __syncthreads();
    }
}

// right-hand side = blockIdx.x (the fast grid index): the CTAs of one block for all
// right-hand sides of a batch are launched together and read the same test-vector lines
// at about the same time, so L2 serves the repeats and DRAM sees each line about once
template <class PF, class PV, typename TC>
__global__ void restrict_kernel(Geom g, Blocking bk, int nvec, const void* __restrict__ vecs,
                                const void* __restrict__ fine, void* coarse) {
    restrict_body<PF, PV, TC>(g, bk, nvec, vecs, (const char*)fine + blockIdx.x * spinor_bytes<PF>(g.V),
                              (char*)coarse + blockIdx.x * (size_t)bk.Vc * 2 * nvec * sizeof(cx<TC>), blockIdx.y,
                              gridDim.y);
}
// ragged batch: bc = R f32 for every problem in one launch (one CTA per block)
template <class PV>
__global__ void restrict_ragged_kernel(const RaggedDev* __restrict__ d, const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    restrict_body<P32, PV, float>(q.g, q.bk, q.nvec, q.vecs, q.f32, q.bc, bx, gx);
}

// ------------------------------------------------------------ prolongation
// One CTA per block, one thread per site: psi'(x) = sum_{s,i} x_c(X, s, i) P_s v_i(x)
// with the loads of a group of test vectors in flight together.
template <class PF, class PV, typename TC>
DEV void prolong_body(const Geom& g, const Blocking& bk, int nvec, const void* __restrict__ vecs,
                      const void* __restrict__ coarse, void* fine, int by, int gy) {
    using T = typename PF::T;
    constexpr int G = kVecGroup<PV>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* xc = reinterpret_cast<cx<T>*>(smem_raw);   // [2*nvec]
    const int nc = 2 * nvec;
    const size_t vb = spinor_bytes<PV>(g.V);
    for (int Xi = by; Xi < bk.Vc; Xi += gy) {
        for (int j = threadIdx.x; j < nc; j += blockDim.x)
            xc[j] = ccast<T>(CStore<TC>::ld(coarse, (size_t)Xi * nc + j));
        __syncthreads();
        const int l = threadIdx.x;
        if (l < bk.Vb) {
            int c[4];
            int s = block_site(g, bk, Xi, l, c);
            cx<T> out[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) out[k] = czero<T>();
            for (int i0 = 0; i0 < nvec; i0 += G) {
                RawSite<PV> raw[G];
#pragma unroll
                for (int u = 0; u < G; ++u)
                    if (i0 + u < nvec) raw[u].load((const char*)vecs + (size_t)(i0 + u) * vb, g.V, s);
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    if (i0 + u >= nvec) break;
                    const cx<T> a0 = xc[i0 + u], a1 = xc[nvec + i0 + u];
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        cfma(out[k], a0, ccast<T>(raw[u].get(k)));
                        cfma(out[6 + k], a1, ccast<T>(raw[u].get(6 + k)));
                    }
                }
            }
            SpinorIO<PF>::store(fine, g.V, s, out);
        }
        __syncthreads();
    }
}

// right-hand side = blockIdx.x, as in restrict_kernel
template <class PF, class PV, typename TC>
__global__ void prolong_kernel(Geom g, Blocking bk, int nvec, const void* __restrict__ vecs,
                               const void* __restrict__ coarse, void* fine) {
    prolong_body<PF, PV, TC>(g, bk, nvec, vecs,
                             (const char*)coarse + blockIdx.x * (size_t)bk.Vc * 2 * nvec * sizeof(cx<TC>),
                             (char*)fine + blockIdx.x * spinor_bytes<PF>(g.V), blockIdx.y, gridDim.y);
}
// ragged batch: z = P xc for every problem in one launch (one CTA per block)
template <class PV>
__global__ void prolong_ragged_kernel(const RaggedDev* __restrict__ d, const int* __restrict__ off, int np) {
    int p, bx, gx;
    ragged_locate(off, np, p, bx, gx);
    const RaggedDev& q = d[p];
    prolong_body<P32, PV, float>(q.g, q.bk, q.nvec, q.vecs, q.xc, q.z, bx, gx);
}

// ------------------------------------------------------------ orthonormalisation
// Per (block, chirality): Gram-Schmidt over i = 0..nvec-1 in index order against
// the previous (orthonormal) vectors, in FP64.  Each projection takes the
// coefficients <v_j, w> of all previous vectors in one pass (classical form:
// per-warp sums into shared memory, one barrier, one cross-warp sum per
// coefficient), then subtracts them in a second pass over the vectors.  A second
// projection follows only if the first removed more than three quarters of
// |w|^2: against an orthonormal set one projection leaves w orthogonal to about
// eps |w0| / |w| <= 2 eps otherwise (the DGKS test).  Either way the result is
// the QR factor with a positive diagonal to rounding, the vectors that
// projecting one vector after another gives.
template <class PV>
__global__ void orthonormalise_kernel(Geom g, Blocking bk, int nvec, void* vecs, int* err) {
    __shared__ double red[3 * 32];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<double>* part = reinterpret_cast<cx<double>*>(smem_raw);   // [nwarps][nvec]
    cx<double>* coef = part + (size_t)(blockDim.x / 32) * nvec;    // [nvec]
    const int Xi = blockIdx.x, chi = blockIdx.y;
    const int l = threadIdx.x, lane = l & 31, warp = l >> 5, nw = blockDim.x >> 5;
    const bool active = l < bk.Vb;
    const size_t vb = spinor_bytes<PV>(g.V);
    int c[4], s = 0;
    if (active) s = block_site(g, bk, Xi, l, c);
    auto load_half = [&](int j, cx<double> (&q)[6]) {
        if (active) {
            cx<typename PV::T> u[12];
            SpinorIO<PV>::load_rw((const char*)vecs + j * vb, g.V, s, u);
#pragma unroll
            for (int k = 0; k < 6; ++k) q[k] = ccast<double>(u[6 * chi + k]);
        } else {
#pragma unroll
            for (int k = 0; k < 6; ++k) q[k] = czero<double>();
        }
    };
    for (int i = 0; i < nvec; ++i) {
        cx<double> w[6];
        load_half(i, w);
        double n0[1] = {0};
        for (int k = 0; k < 6; ++k) n0[0] += norm2(w[k]);
        block_sum<double, 1>(n0, red);
        for (int pass = 0; pass < 2 && i > 0; ++pass) {
            if (pass == 1) {   // a second projection only after a large cancellation
                double n1[1] = {0};
                for (int k = 0; k < 6; ++k) n1[0] += norm2(w[k]);
                block_sum<double, 1>(n1, red);
                if (n1[0] > 0.25 * n0[0]) break;
            }
            for (int j = 0; j < i; ++j) {
                cx<double> q[6];
                load_half(j, q);
                cx<double> d = czero<double>();
#pragma unroll
                for (int k = 0; k < 6; ++k) d = d + cmulc(q[k], w[k]);
                d.re = warp_sum(d.re);
                d.im = warp_sum(d.im);
                if (lane == 0) part[warp * nvec + j] = d;
            }
            __syncthreads();
            for (int j = l; j < i; j += blockDim.x) {
                cx<double> t = czero<double>();
                for (int ww = 0; ww < nw; ++ww) t = t + part[ww * nvec + j];
                coef[j] = t;
            }
            __syncthreads();
            for (int j = 0; j < i; ++j) {
                cx<double> q[6];
                load_half(j, q);
                const cx<double> cc = coef[j];
#pragma unroll
                for (int k = 0; k < 6; ++k) w[k] = w[k] - cc * q[k];
            }
            __syncthreads();   // part / coef are rewritten by the next pass
        }
        double nn[1] = {0};
        for (int k = 0; k < 6; ++k) nn[0] += norm2(w[k]);
        block_sum<double, 1>(nn, red);
        // rank test: |w| <= 1e-12 |w0| (FP64 storage), 1e-5 |w0| (FP32 storage)
        const double rtol2 = PV::id == 0 ? 1e-24 : 1e-10;
        if (!(nn[0] > rtol2 * n0[0])) {
            if (threadIdx.x == 0) atomicExch(err, 1);
            nn[0] = 1.0;
        }
        double inv = 1.0 / sqrt(nn[0]);
        if (active) {
            // the other chirality half belongs to the CTA (Xi, 1 - chi): write ours only
            cx<typename PV::T> hv[6];
            for (int k = 0; k < 6; ++k) hv[k] = ccast<typename PV::T>(inv * w[k]);
            SpinorIO<PV>::store_half((char*)vecs + i * vb, g.V, s, chi, hv);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ Galerkin operator
// CTA (block Xi, pair of columns J = (t, j)): for every direction d the fields
// T_d = H_d P_t v_j on the sites of Xi (H_0 = D_SAP on the block, H_{+-mu} =
// the hops of D leaving Xi through its +-mu face) are formed for both columns
// and projected on all basis vectors of Xi: B[Xi][I][d][J] = <Xi, I| T_d>.
// Each test-vector load serves both columns; in a face direction only the
// face sites of the block (a quarter of them for 4^4 blocks) load anything,
// and a warp without face sites skips the direction; the four projections of
// a vector (two columns x two chiralities) are summed over the warp by one
// transposed shuffle reduction.
template <class PV, typename TC>
__global__ void galerkin_kernel(Geom g, Blocking bk, int nvec, const void* __restrict__ vecs,
                                const void* __restrict__ U, const void* __restrict__ C, typename PV::T kappa,
                                void* B) {
    using T = typename PV::T;
    constexpr int NQ = 8;   // per vector: column a / b x chirality 0 / 1 x (re, im)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nc = 2 * nvec;
    T* partf = reinterpret_cast<T*>(smem_raw);   // [nwarps][2 columns][nc] complex
    cx<T>* part = reinterpret_cast<cx<T>*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int Xi = blockIdx.x, Ja = 2 * blockIdx.y, Jb = Ja + 1;
    const bool hasB = Jb < nc;
    const int ta = Ja / nvec, ja = Ja % nvec, tb = hasB ? Jb / nvec : 0, jb = hasB ? Jb % nvec : 0;
    const size_t vb = spinor_bytes<PV>(g.V);
    const char* va = (const char*)vecs + ja * vb;
    const char* vbp = (const char*)vecs + jb * vb;
    const int l = threadIdx.x;
    const bool active = l < bk.Vb;
    const int qi = transposed_index<NQ>(lane);
    const bool writer = (lane & (32 / NQ - 1)) == 0;
    int c[4] = {0, 0, 0, 0}, lc[4] = {0, 0, 0, 0}, s = 0;
    if (active) {
        s = block_site(g, bk, Xi, l, c);
        for (int mu = 0; mu < 4; ++mu) lc[mu] = c[mu] % bk.b[mu];
    }
    auto load_proj = [&](const char* v, int t, int site, cx<T> out[12]) {
        SpinorIO<PV>::load(v, g.V, site, out);
#pragma unroll
        for (int k = 0; k < 6; ++k) out[6 * (1 - t) + k] = czero<T>();
    };
    // acc_a += coeff (1 - dir gamma_mu) W P_ta v_ja(n), acc_b likewise (one link load)
    auto hop2 = [&](int n, int linksite, int mu, int dir, T coeff, cx<T> (&acc_a)[12], cx<T> (&acc_b)[12]) {
        cx<T> psi[12], u[3][3];
        GaugeIO<PV>::load(U, g.V, mu, linksite, u);
        load_proj(va, ta, n, psi);
        hop_accum<T>(acc_a, psi, u, mu, dir, coeff);
        if (hasB) {
            load_proj(vbp, tb, n, psi);
            hop_accum<T>(acc_b, psi, u, mu, dir, coeff);
        }
    };
    for (int d = 0; d < 9; ++d) {
        const int mu = d == 0 ? 0 : (d - 1) % 4;
        const int dir = d <= 4 ? +1 : -1;
        const bool face = d == 0 || (dir > 0 ? (lc[mu] == bk.b[mu] - 1) : (lc[mu] == 0));
        const bool work = active && face;
        cx<T> Ta[12], Tb[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) Ta[k] = Tb[k] = czero<T>();
        if (work) {
            float ph;
            if (d == 0) {
                cx<T> psi[12];
                load_proj(va, ta, s, psi);
                clover_apply<PV>(C, g.V, s, psi, Ta);
                if (hasB) {
                    load_proj(vbp, tb, s, psi);
                    clover_apply<PV>(C, g.V, s, psi, Tb);
                }
                for (int m = 0; m < 4; ++m) {
                    if (lc[m] != bk.b[m] - 1) {
                        int n = neighbour(g, s, c, m, +1, ph);
                        hop2(n, s, m, +1, -kappa * T(ph), Ta, Tb);
                    }
                    if (lc[m] != 0) {
                        int n = neighbour(g, s, c, m, -1, ph);
                        hop2(n, n, m, -1, -kappa * T(ph), Ta, Tb);
                    }
                }
            } else {
                int n = neighbour(g, s, c, mu, dir, ph);
                hop2(n, dir > 0 ? s : n, mu, dir, -kappa * T(ph), Ta, Tb);
            }
        }
        const bool wwork = __any_sync(0xffffffffu, work);
        for (int i = 0; i < nvec; ++i) {
            if (!wwork) {   // no face site in this warp: its partial sums are zero
                if (lane < 4) part[(warp * 2 + (lane >> 1)) * nc + (lane & 1) * nvec + i] = czero<T>();
                continue;
            }
            cx<T> d0a = czero<T>(), d1a = czero<T>(), d0b = czero<T>(), d1b = czero<T>();
            if (work) {
                cx<T> v[12];
                SpinorIO<PV>::load((const char*)vecs + i * vb, g.V, s, v);
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    cfmac(d0a, v[k], Ta[k]);
                    cfmac(d1a, v[6 + k], Ta[6 + k]);
                    cfmac(d0b, v[k], Tb[k]);
                    cfmac(d1b, v[6 + k], Tb[6 + k]);
                }
            }
            T q[NQ] = {d0a.re, d0a.im, d1a.re, d1a.im, d0b.re, d0b.im, d1b.re, d1b.im};
            const T tot = transposed_warp_sum<NQ>(q, lane);
            if (writer) {
                const int col = qi >> 2, comp = qi & 3;
                const int row = (comp < 2 ? 0 : nvec) + i;
                partf[2 * ((warp * 2 + col) * nc + row) + (comp & 1)] = tot;
            }
        }
        __syncthreads();
        for (int r = threadIdx.x; r < 2 * nc; r += blockDim.x) {
            const int col = r / nc, row = r % nc;
            if (col == 1 && !hasB) continue;
            cx<T> acc = czero<T>();
            for (int w = 0; w < nw; ++w) acc = acc + part[(w * 2 + col) * nc + row];
            CStore<TC>::st(B, (((size_t)Xi * nc + row) * 9 + d) * nc + (col ? Jb : Ja), ccast<TC>(acc));
        }
        __syncthreads();
    }
}

int threads_for(const Blocking& bk) { return (bk.Vb + 31) / 32 * 32; }

template <class PF, class PV, typename TC>
cudaError_t restrict_impl(const GeomH& gh, const BlockH& bh, int nvec, const void* vecs, const void* fine,
                          void* coarse, int nrhs, cudaStream_t st) {
    Geom g = make_geom(gh);
    Blocking bk = make_blocking(gh, bh);
    int th = threads_for(bk);
    size_t smem = (size_t)(th / 32) * 2 * nvec * sizeof(cx<typename PF::T>);
    (note_launch(), restrict_kernel<PF, PV, TC><<<dim3(nrhs, std::min(bk.Vc, 65535)), th, smem, st>>>(g, bk, nvec, vecs,
                                                                                                 fine, coarse));
    return cudaGetLastError();
}
template <class PF, class PV, typename TC>
cudaError_t prolong_impl(const GeomH& gh, const BlockH& bh, int nvec, const void* vecs, const void* coarse,
                         void* fine, int nrhs, cudaStream_t st) {
    Geom g = make_geom(gh);
    Blocking bk = make_blocking(gh, bh);
    int th = threads_for(bk);
    size_t smem = (size_t)2 * nvec * sizeof(cx<typename PF::T>);
    (note_launch(), prolong_kernel<PF, PV, TC><<<dim3(nrhs, std::min(bk.Vc, 65535)), th, smem, st>>>(g, bk, nvec, vecs,
                                                                                                coarse, fine));
    return cudaGetLastError();
}

}  // namespace

#define DISPATCH_F(fprec, ...)                 \
    if (fprec == 0) { using PF = P64; __VA_ARGS__; } \
    else if (fprec == 1) { using PF = P32; __VA_ARGS__; } \
    else { using PF = P16; __VA_ARGS__; }

cudaError_t launch_restrict_fine(int fprec, int vprec, int cprec, const GeomH& g, const BlockH& bk, int nvec,
                                 const void* vecs, const void* fine, void* coarse, int nrhs, cudaStream_t st) {
    if (vprec == 0) {
        if (cprec == 0) { DISPATCH_F(fprec, return restrict_impl<PF, P64, double>(g, bk, nvec, vecs, fine, coarse, nrhs, st)); }
        DISPATCH_F(fprec, return restrict_impl<PF, P64, float>(g, bk, nvec, vecs, fine, coarse, nrhs, st));
    }
    if (vprec == 2) {   // half-precision test vectors with a per-site scale
        if (cprec == 0) { DISPATCH_F(fprec, return restrict_impl<PF, P16, double>(g, bk, nvec, vecs, fine, coarse, nrhs, st)); }
        DISPATCH_F(fprec, return restrict_impl<PF, P16, float>(g, bk, nvec, vecs, fine, coarse, nrhs, st));
    }
    if (cprec == 0) { DISPATCH_F(fprec, return restrict_impl<PF, P32, double>(g, bk, nvec, vecs, fine, coarse, nrhs, st)); }
    DISPATCH_F(fprec, return restrict_impl<PF, P32, float>(g, bk, nvec, vecs, fine, coarse, nrhs, st));
}
cudaError_t launch_prolong_fine(int fprec, int vprec, int cprec, const GeomH& g, const BlockH& bk, int nvec,
                                const void* vecs, const void* coarse, void* fine, int nrhs, cudaStream_t st) {
    if (vprec == 0) {
        if (cprec == 0) { DISPATCH_F(fprec, return prolong_impl<PF, P64, double>(g, bk, nvec, vecs, coarse, fine, nrhs, st)); }
        DISPATCH_F(fprec, return prolong_impl<PF, P64, float>(g, bk, nvec, vecs, coarse, fine, nrhs, st));
    }
    if (vprec == 2) {
        if (cprec == 0) { DISPATCH_F(fprec, return prolong_impl<PF, P16, double>(g, bk, nvec, vecs, coarse, fine, nrhs, st)); }
        DISPATCH_F(fprec, return prolong_impl<PF, P16, float>(g, bk, nvec, vecs, coarse, fine, nrhs, st));
    }
    if (cprec == 0) { DISPATCH_F(fprec, return prolong_impl<PF, P32, double>(g, bk, nvec, vecs, coarse, fine, nrhs, st)); }
    DISPATCH_F(fprec, return prolong_impl<PF, P32, float>(g, bk, nvec, vecs, coarse, fine, nrhs, st));
}
cudaError_t launch_orthonormalise_fine(int vprec, const GeomH& gh, const BlockH& bh, int nvec, void* vecs,
                                       int* err, cudaStream_t st) {
    Geom g = make_geom(gh);
    Blocking bk = make_blocking(gh, bh);
    dim3 grid(bk.Vc, 2);
    int th = threads_for(bk);
    const size_t smem = ((size_t)(th / 32) + 1) * nvec * sizeof(cx<double>);
    if (vprec == 0) (note_launch(), orthonormalise_kernel<P64><<<grid, th, smem, st>>>(g, bk, nvec, vecs, err));
    else (note_launch(), orthonormalise_kernel<P32><<<grid, th, smem, st>>>(g, bk, nvec, vecs, err));
    return cudaGetLastError();
}
cudaError_t launch_galerkin_fine(int vprec, int cprec, const GeomH& gh, const BlockH& bh, int nvec, const void* vecs,
                                 const void* U, const void* C, double kappa, void* B, cudaStream_t st) {
    Geom g = make_geom(gh);
    Blocking bk = make_blocking(gh, bh);
    int th = threads_for(bk);
    dim3 grid(bk.Vc, nvec);   // pairs of columns
    if (vprec == 0) {
        size_t smem = (size_t)(th / 32) * 2 * 2 * nvec * sizeof(cx<double>);
        if (cprec == 0) (note_launch(), galerkin_kernel<P64, double><<<grid, th, smem, st>>>(g, bk, nvec, vecs, U, C, kappa, B));
        else (note_launch(), galerkin_kernel<P64, float><<<grid, th, smem, st>>>(g, bk, nvec, vecs, U, C, kappa, B));
    } else {
        size_t smem = (size_t)(th / 32) * 2 * 2 * nvec * sizeof(cx<float>);
        if (cprec == 0) (note_launch(), galerkin_kernel<P32, double><<<grid, th, smem, st>>>(g, bk, nvec, vecs, U, C, (float)kappa, B));
        else (note_launch(), galerkin_kernel<P32, float><<<grid, th, smem, st>>>(g, bk, nvec, vecs, U, C, (float)kappa, B));
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- ragged batches
// blockDim: the largest problem's block, rounded up to whole warps; shared memory for that many warps
cudaError_t launch_restrict_ragged(int vprec, const void* d, const int* off, int np, int ctas, int max_vb, int max_nvec,
                                   cudaStream_t st) {
    const int th = (max_vb + 31) / 32 * 32;
    const size_t smem = (size_t)(th / 32) * 2 * max_nvec * sizeof(cx<float>);
    const RaggedDev* dd = (const RaggedDev*)d;
    if (vprec == 0) (note_launch(), restrict_ragged_kernel<P64><<<ctas, th, smem, st>>>(dd, off, np));
    else if (vprec == 1) (note_launch(), restrict_ragged_kernel<P32><<<ctas, th, smem, st>>>(dd, off, np));
    else (note_launch(), restrict_ragged_kernel<P16><<<ctas, th, smem, st>>>(dd, off, np));
    return cudaGetLastError();
}
cudaError_t launch_prolong_ragged(int vprec, const void* d, const int* off, int np, int ctas, int max_vb, int max_nvec,
                                  cudaStream_t st) {
    const int th = (max_vb + 31) / 32 * 32;
    const size_t smem = (size_t)2 * max_nvec * sizeof(cx<float>);
    const RaggedDev* dd = (const RaggedDev*)d;
    if (vprec == 0) (note_launch(), prolong_ragged_kernel<P64><<<ctas, th, smem, st>>>(dd, off, np));
    else if (vprec == 1) (note_launch(), prolong_ragged_kernel<P32><<<ctas, th, smem, st>>>(dd, off, np));
    else (note_launch(), prolong_ragged_kernel<P16><<<ctas, th, smem, st>>>(dd, off, np));
    return cudaGetLastError();
}
