// Multigrid kernels on coarse lattices, used when the hierarchy has three or
// more grids: restriction and prolongation from level l >= 1 to l+1 (Eqs. 5-6
// with the chirality halves of the coarse dof axis), block Gram-Schmidt of the
// level-l test vectors, the Galerkin stencil of level l+1 built from the
// 9-point stencil of level l (Eq. 7), and the SAP half sweep with
// minimal-residual domain solves on a coarse lattice (Sec. 3 listing).
//
// Layouts: coarse vectors [site][nc] complex; test vectors [nvec][site][nc];
// stencils [X][row][d][col] (d = 0 self, 1+mu forward, 5+mu backward).
#include "common.cuh"
#include "kernels.h"

namespace {

// a coarse lattice together with its blocking into the domains of the next level
struct CB {
    int L[4];
    int V;
    int b[4];
    int C[4];
    int Vb, Vc;
};

CB make_cb(const GeomH& g, const BlockH& bh) {
    CB k;
    k.V = g.V;
    k.Vb = 1;
    k.Vc = 1;
    for (int mu = 0; mu < 4; ++mu) {
        k.L[mu] = g.L[mu];
        k.b[mu] = bh.b[mu];
        k.C[mu] = g.L[mu] / bh.b[mu];
        k.Vb *= k.b[mu];
        k.Vc *= k.C[mu];
    }
    return k;
}

DEV void unflatten(int i, const int n[4], int c[4]) {
    c[0] = i % n[0];
    i /= n[0];
    c[1] = i % n[1];
    i /= n[1];
    c[2] = i % n[2];
    c[3] = i / n[2];
}
DEV int flatten(const int c[4], const int n[4]) { return c[0] + n[0] * (c[1] + n[1] * (c[2] + n[2] * c[3])); }

// lattice site of local site l of block Xi, with its local coordinates
DEV int cb_site(const CB& k, int Xi, int l, int lc[4]) {
    int X[4], c[4];
    unflatten(Xi, k.C, X);
    unflatten(l, k.b, lc);
    for (int mu = 0; mu < 4; ++mu) c[mu] = X[mu] * k.b[mu] + lc[mu];
    return flatten(c, k.L);
}
// neighbour of site s in stencil direction d (periodic)
DEV int cb_nbr(const CB& k, int s, int d) {
    if (d == 0) return s;
    int c[4];
    unflatten(s, k.L, c);
    const int mu = (d - 1) & 3;
    c[mu] = d <= 4 ? (c[mu] + 1 == k.L[mu] ? 0 : c[mu] + 1) : (c[mu] == 0 ? k.L[mu] - 1 : c[mu] - 1);
    return flatten(c, k.L);
}
// does the hop d from a site with local coordinates lc stay inside its block?
DEV bool stays(const CB& k, const int lc[4], int d) {
    if (d == 0) return true;
    const int mu = (d - 1) & 3;
    return d <= 4 ? lc[mu] != k.b[mu] - 1 : lc[mu] != 0;
}
// block Xi of the given colour: the k-th block with (sum of block coordinates) % 2 == colour
DEV int colour_block(const CB& k, int idx, int colour) {
    const int h0 = k.C[0] / 2;
    int rest = idx / h0;
    const int X1 = rest % k.C[1];
    rest /= k.C[1];
    const int X2 = rest % k.C[2];
    const int X3 = rest / k.C[2];
    const int X0 = 2 * (idx % h0) + ((X1 + X2 + X3 + colour) & 1);
    return X0 + k.C[0] * (X1 + k.C[1] * (X2 + k.C[2] * X3));
}

template <typename TC> DEV cx<TC> ldv(const void* p, size_t i);
template <> DEV cx<double> ldv<double>(const void* p, size_t i) {
    double2 t = ((const double2*)p)[i];
    return {t.x, t.y};
}
template <> DEV cx<float> ldv<float>(const void* p, size_t i) {
    float2 t = ((const float2*)p)[i];
    return {t.x, t.y};
}
template <typename TC> DEV void stv(void* p, size_t i, cx<TC> v);
template <> DEV void stv<double>(void* p, size_t i, cx<double> v) { ((double2*)p)[i] = make_double2(v.re, v.im); }
template <> DEV void stv<float>(void* p, size_t i, cx<float> v) { ((float2*)p)[i] = make_float2(v.re, v.im); }

// operator entry i: complex in TC, or a bfloat16 pair (BF) widened to FP32
template <typename TC, bool BF> DEV cx<TC> ldop(const void* B, size_t i) { return ldv<TC>(B, i); }
template <> DEV cx<float> ldop<float, true>(const void* B, size_t i) {
    float2 f = __bfloat1622float2(((const __nv_bfloat162*)B)[i]);
    return {f.x, f.y};
}

// ------------------------------------------------------------ Eq. 5
// out(X, s*nv + i) = sum_{x in X} sum_{a in half s} conj(v_i(x)[a]) in(x)[a]
// grid (Vc, nrhs); a warp per output, lanes over the block's terms
template <typename TC>
__global__ void crestrict_kernel(CB k, int nc, int nv, const void* __restrict__ vecs, const void* __restrict__ in,
                                 void* out) {
    const int Xi = blockIdx.x, r = blockIdx.y;
    const int half = nc / 2, nt = k.Vb * half;
    const size_t vs = (size_t)k.V * nc;
    const char* xin = (const char*)in + (size_t)r * vs * sizeof(cx<TC>);
    char* y = (char*)out + (size_t)r * k.Vc * 2 * nv * sizeof(cx<TC>);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = warp; o < 2 * nv; o += nw) {
        const int s = o / nv, i = o % nv;
        cx<TC> acc = czero<TC>();
        for (int t = lane; t < nt; t += 32) {
            int lc[4];
            const size_t e = (size_t)cb_site(k, Xi, t / half, lc) * nc + s * half + t % half;
            acc = acc + cmulc(ldv<TC>(vecs, i * vs + e), ldv<TC>(xin, e));
        }
        acc.re = warp_sum(acc.re);
        acc.im = warp_sum(acc.im);
        if (lane == 0) stv<TC>(y, (size_t)Xi * 2 * nv + o, acc);
    }
}

// ------------------------------------------------------------ Eq. 6
// out(x)[a] = sum_i v_i(x)[a] in(X(x), s(a)*nv + i); grid (Vc, nrhs)
template <typename TC>
__global__ void cprolong_kernel(CB k, int nc, int nv, const void* __restrict__ vecs, const void* __restrict__ in,
                                void* out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<TC>* xc = reinterpret_cast<cx<TC>*>(smem_raw);   // [2 nv]
    const int Xi = blockIdx.x, r = blockIdx.y;
    const int half = nc / 2;
    const size_t vs = (size_t)k.V * nc;
    const char* cin = (const char*)in + (size_t)r * k.Vc * 2 * nv * sizeof(cx<TC>);
    char* y = (char*)out + (size_t)r * vs * sizeof(cx<TC>);
    for (int o = threadIdx.x; o < 2 * nv; o += blockDim.x) xc[o] = ldv<TC>(cin, (size_t)Xi * 2 * nv + o);
    __syncthreads();
    for (int t = threadIdx.x; t < k.Vb * nc; t += blockDim.x) {
        int lc[4];
        const int a = t % nc, s = a / half;
        const size_t e = (size_t)cb_site(k, Xi, t / nc, lc) * nc + a;
        cx<TC> acc = czero<TC>();
        for (int i = 0; i < nv; ++i) acc = acc + ldv<TC>(vecs, i * vs + e) * xc[s * nv + i];
        stv<TC>(y, e, acc);
    }
}

// ------------------------------------------------------------ block Gram-Schmidt
// Per (block, chirality): i = 0..nv-1 in index order, each vector projected
// against the previous ones twice (one block reduction per projection), FP64
// arithmetic whatever the storage.  EPT elements of the block's chirality
// half per thread.
template <typename TC, int EPT>
__global__ void cortho_kernel(CB k, int nc, int nv, void* vecs, int* err) {
    __shared__ double red[2 * 32];
    const int Xi = blockIdx.x, chi = blockIdx.y;
    const int half = nc / 2, E = k.Vb * half;
    const size_t vs = (size_t)k.V * nc;
    size_t idx[EPT];
    bool act[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int t = threadIdx.x + e * blockDim.x;
        act[e] = t < E;
        idx[e] = 0;
        if (act[e]) {
            int lc[4];
            idx[e] = (size_t)cb_site(k, Xi, t / half, lc) * nc + chi * half + t % half;
        }
    }
    for (int i = 0; i < nv; ++i) {
        cx<double> w[EPT];
        double n0[1] = {0};
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            w[e] = act[e] ? ccast<double>(ldv<TC>(vecs, i * vs + idx[e])) : czero<double>();
            n0[0] += norm2(w[e]);
        }
        block_sum<double, 1>(n0, red);
        for (int pass = 0; pass < 2; ++pass) {
            for (int j = 0; j < i; ++j) {
                cx<double> q[EPT];
                double d[2] = {0, 0};
#pragma unroll
                for (int e = 0; e < EPT; ++e) {
                    q[e] = act[e] ? ccast<double>(ldv<TC>(vecs, j * vs + idx[e])) : czero<double>();
                    const cx<double> t = cmulc(q[e], w[e]);
                    d[0] += t.re;
                    d[1] += t.im;
                }
                block_sum<double, 2>(d, red);
                const cx<double> c = {d[0], d[1]};
#pragma unroll
                for (int e = 0; e < EPT; ++e) w[e] = w[e] - c * q[e];
            }
        }
        double nn[1] = {0};
#pragma unroll
        for (int e = 0; e < EPT; ++e) nn[0] += norm2(w[e]);
        block_sum<double, 1>(nn, red);
        // rank test: |w| <= 1e-12 |w0| (FP64 storage), 1e-5 |w0| (FP32 storage)
        const double rtol2 = sizeof(TC) == 8 ? 1e-24 : 1e-10;
        if (!(nn[0] > rtol2 * n0[0])) {
            if (threadIdx.x == 0) atomicExch(err, 1);
            nn[0] = 1.0;
        }
        const double inv = 1.0 / sqrt(nn[0]);
#pragma unroll
        for (int e = 0; e < EPT; ++e)
            if (act[e]) stv<TC>(vecs, i * vs + idx[e], ccast<TC>(inv * w[e]));
    }
}

// ------------------------------------------------------------ Eq. 7 on a coarse level
// Bout[X][I][d][J] = sum over the hops x -> x+d1 of level l that couple block X
// to block X+d of  conj(v_I(x)) . B_l[x][d1] . v_J(x+d1),
// v_I = P_s v_i (I = s*nv + i).  d = 0 collects d1 = 0 and the hops that stay
// in X; d = +-mu the hops that leave X across its +-mu face.  grid (Vc, 9).
template <typename TC, typename TO>
__global__ void cgalerkin_kernel(CB k, int nc, int nv, const void* __restrict__ vecs, const void* __restrict__ B,
                                 void* Bout) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nco = 2 * nv, half = nc / 2;
    cx<TC>* Vx = reinterpret_cast<cx<TC>*>(smem_raw);   // [nc][nv]
    cx<TC>* Vy = Vx + nc * nv;                            // [nc][nv]
    cx<TC>* Bm = Vy + nc * nv;                            // [nc][nc]
    cx<TC>* T = Bm + nc * nc;                             // [nc][nco]
    constexpr int kMaxOut = 16;                           // nco * nco <= 16 * blockDim
    const int Xi = blockIdx.x, d = blockIdx.y;
    const size_t vs = (size_t)k.V * nc;
    cx<TC> acc[kMaxOut];
#pragma unroll
    for (int m = 0; m < kMaxOut; ++m) acc[m] = czero<TC>();
    for (int l = 0; l < k.Vb; ++l) {
        int lc[4];
        const int x = cb_site(k, Xi, l, lc);
        for (int d1 = 0; d1 < 9; ++d1) {
            bool use;
            if (d == 0) use = stays(k, lc, d1);
            else use = d1 == d && !stays(k, lc, d1);
            if (!use) continue;   // uniform over the CTA
            const int y = cb_nbr(k, x, d1);
            __syncthreads();
            for (int t = threadIdx.x; t < nc * nv; t += blockDim.x) {
                const int a = t / nv, i = t % nv;
                Vx[t] = ldv<TC>(vecs, i * vs + (size_t)x * nc + a);
                Vy[t] = ldv<TC>(vecs, i * vs + (size_t)y * nc + a);
            }
            for (int t = threadIdx.x; t < nc * nc; t += blockDim.x) {
                const int a = t / nc, b = t % nc;
                Bm[t] = ldv<TC>(B, (((size_t)x * nc + a) * 9 + d1) * nc + b);
            }
            __syncthreads();
            // T[a][J] = sum_{b in half t(J)} Bm[a][b] v_j(y)[b]
            for (int t = threadIdx.x; t < nc * nco; t += blockDim.x) {
                const int a = t / nco, J = t % nco, tj = J / nv, j = J % nv;
                cx<TC> s = czero<TC>();
                for (int b = tj * half; b < (tj + 1) * half; ++b) s = s + Bm[a * nc + b] * Vy[b * nv + j];
                T[t] = s;
            }
            __syncthreads();
#pragma unroll
            for (int m = 0; m < kMaxOut; ++m) {
                const int o = threadIdx.x + m * blockDim.x;
                if (o < nco * nco) {
                    const int I = o / nco, J = o % nco, si = I / nv, i = I % nv;
                    cx<TC> s = czero<TC>();
                    for (int a = si * half; a < (si + 1) * half; ++a) s = s + cmulc(Vx[a * nv + i], T[a * nco + J]);
                    acc[m] = acc[m] + s;
                }
            }
        }
    }
#pragma unroll
    for (int m = 0; m < kMaxOut; ++m) {
        const int o = threadIdx.x + m * blockDim.x;
        if (o < nco * nco) {
            const int I = o / nco, J = o % nco;
            stv<TO>(Bout, (((size_t)Xi * nco + I) * 9 + d) * nco + J, ccast<TO>(acc[m]));
        }
    }
}

// ------------------------------------------------------------ SAP on a coarse level
// One CTA per domain of the given colour (domains = blocks of this level),
// blockIdx.y = right-hand side.  r = b - D x on the domain (x_mode as for the
// fine kernel: 0 iterate everywhere, 1 x = 0, 2 x = 0 on the active domains),
// nmr minimal-residual steps on D restricted to the domain (in-domain hops
// only), x = z (+ x).  Rows are computed a warp at a time (lanes over the
// contiguous 9 * nc run of a stencil row); domain vectors live in shared memory.
template <typename TC, bool BF>
__global__ void __launch_bounds__(1024) csap_half_kernel(CB k, int nc, int colour, int nmr, int x_mode, const void* __restrict__ B,
                                 const void* __restrict__ b, void* x) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = k.Vb * nc;
    cx<TC>* rs = reinterpret_cast<cx<TC>*>(smem_raw);   // [n] residual
    cx<TC>* zs = rs + n;                                  // [n] correction
    cx<TC>* As = zs + n;                                  // [n] D_SAP r
    TC* red = reinterpret_cast<TC*>(As + n);              // [3][32]
    const int Xi = colour_block(k, blockIdx.x, colour);
    const size_t off = (size_t)blockIdx.y * k.V * nc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int lstr[4] = {1, k.b[0], k.b[0] * k.b[1], k.b[0] * k.b[1] * k.b[2]};
    // residual on the domain
    for (int row = warp; row < n; row += nw) {
        const int l = row / nc, a = row % nc;
        int lc[4];
        const int s = cb_site(k, Xi, l, lc);
        cx<TC> acc = czero<TC>();
        if (x_mode != 1) {
            for (int d1 = 0; d1 < 9; ++d1) {
                if (x_mode == 2 && stays(k, lc, d1)) continue;
                const size_t yb = off + (size_t)cb_nbr(k, s, d1) * nc;
                const size_t rb = (((size_t)s * nc + a) * 9 + d1) * nc;
                for (int c = lane; c < nc; c += 32) acc = acc + ldop<TC, BF>(B, rb + c) * ldv<TC>(x, yb + c);
            }
            acc.re = warp_sum(acc.re);
            acc.im = warp_sum(acc.im);
        }
        if (lane == 0) {
            rs[row] = ldv<TC>(b, off + (size_t)s * nc + a) - acc;
            zs[row] = czero<TC>();
        }
    }
    for (int it = 0; it < nmr; ++it) {
        __syncthreads();
        for (int row = warp; row < n; row += nw) {
            const int l = row / nc, a = row % nc;
            int lc[4];
            const int s = cb_site(k, Xi, l, lc);
            cx<TC> acc = czero<TC>();
            for (int d1 = 0; d1 < 9; ++d1) {
                if (!stays(k, lc, d1)) continue;
                const int mu = (d1 - 1) & 3;
                const int ln = d1 == 0 ? l : (d1 <= 4 ? l + lstr[mu] : l - lstr[mu]);
                const size_t rb = (((size_t)s * nc + a) * 9 + d1) * nc;
                for (int c = lane; c < nc; c += 32) acc = acc + ldop<TC, BF>(B, rb + c) * rs[ln * nc + c];
            }
            acc.re = warp_sum(acc.re);
            acc.im = warp_sum(acc.im);
            if (lane == 0) As[row] = acc;
        }
        __syncthreads();
        TC part[3] = {TC(0), TC(0), TC(0)};
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const cx<TC> t = cmulc(As[e], rs[e]);
            part[0] += t.re;
            part[1] += t.im;
            part[2] += norm2(As[e]);
        }
        block_sum<TC, 3>(part, red);
        cx<TC> alpha = czero<TC>();
        if (part[2] > TC(0)) alpha = {part[0] / part[2], part[1] / part[2]};
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            zs[e] = zs[e] + alpha * rs[e];
            rs[e] = rs[e] - alpha * As[e];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        int lc[4];
        const size_t i = off + (size_t)cb_site(k, Xi, e / nc, lc) * nc + e % nc;
        cx<TC> v = zs[e];
        if (x_mode == 0) v = v + ldv<TC>(x, i);
        stv<TC>(x, i, v);
    }
}

int threads_for(int n) {
    int t = (n + 31) / 32 * 32;
    return t < 64 ? 64 : (t > 1024 ? 1024 : t);
}

}  // namespace

cudaError_t launch_restrict_coarse(int vprec, const GeomH& g, const BlockH& bh, int nc, int nvec, const void* vecs,
                                   const void* fine, void* coarse, int nrhs, cudaStream_t st) {
    CB k = make_cb(g, bh);
    dim3 grid(k.Vc, nrhs);
    if (vprec == 0) (note_launch(), crestrict_kernel<double><<<grid, 256, 0, st>>>(k, nc, nvec, vecs, fine, coarse));
    else (note_launch(), crestrict_kernel<float><<<grid, 256, 0, st>>>(k, nc, nvec, vecs, fine, coarse));
    return cudaGetLastError();
}

cudaError_t launch_prolong_coarse(int vprec, const GeomH& g, const BlockH& bh, int nc, int nvec, const void* vecs,
                                  const void* coarse, void* fine, int nrhs, cudaStream_t st) {
    CB k = make_cb(g, bh);
    dim3 grid(k.Vc, nrhs);
    const int th = threads_for(k.Vb * nc);
    if (vprec == 0)
        (note_launch(), cprolong_kernel<double><<<grid, th, 2 * nvec * sizeof(cx<double>), st>>>(k, nc, nvec, vecs, coarse, fine));
    else
        (note_launch(), cprolong_kernel<float><<<grid, th, 2 * nvec * sizeof(cx<float>), st>>>(k, nc, nvec, vecs, coarse, fine));
    return cudaGetLastError();
}

cudaError_t launch_orthonormalise_coarse(int vprec, const GeomH& g, const BlockH& bh, int nc, int nvec, void* vecs,
                                         int* err, cudaStream_t st) {
    CB k = make_cb(g, bh);
    const int E = k.Vb * (nc / 2);
    const int th = threads_for(E);
    const int ept = (E + th - 1) / th;
    if (ept > 4 || nc % 2 != 0) return cudaErrorInvalidValue;
    dim3 grid(k.Vc, 2);
#define CORTHO(T, N) (note_launch(), cortho_kernel<T, N><<<grid, th, 0, st>>>(k, nc, nvec, vecs, err))
    if (vprec == 0) {
        if (ept == 1) CORTHO(double, 1);
        else if (ept == 2) CORTHO(double, 2);
        else CORTHO(double, 4);
    } else {
        if (ept == 1) CORTHO(float, 1);
        else if (ept == 2) CORTHO(float, 2);
        else CORTHO(float, 4);
    }
#undef CORTHO
    return cudaGetLastError();
}

cudaError_t launch_galerkin_coarse(int vprec, int oprec, const GeomH& g, const BlockH& bh, int nc, int nvec,
                                   const void* vecs, const void* B, void* Bout, cudaStream_t st) {
    CB k = make_cb(g, bh);
    const int th = 256;
    if (4 * nvec * nvec > 16 * th || nc % 2 != 0) return cudaErrorInvalidValue;
    dim3 grid(k.Vc, 9);
    const size_t elems = (size_t)2 * nc * nvec + (size_t)nc * nc + (size_t)nc * 2 * nvec;
    if (vprec == 0) {
        const size_t smem = elems * sizeof(cx<double>);
        cudaError_t e = cudaFuncSetAttribute(cgalerkin_kernel<double, double>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        (note_launch(), cgalerkin_kernel<double, double><<<grid, th, smem, st>>>(k, nc, nvec, vecs, B, Bout));
    } else {
        // FP32 level; the next level's stencil is stored in FP32 or (oprec 0) widened to FP64
        const size_t smem = elems * sizeof(cx<float>);
        auto fn = oprec == 0 ? cgalerkin_kernel<float, double> : cgalerkin_kernel<float, float>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        (note_launch(), fn<<<grid, th, smem, st>>>(k, nc, nvec, vecs, B, Bout));
    }
    return cudaGetLastError();
}

cudaError_t launch_coarse_sap_half(int kprec, const GeomH& g, const BlockH& bh, int nc, int colour, int nmr,
                                   int x_mode, const void* B, const void* b, void* x, int nrhs, cudaStream_t st) {
    CB k = make_cb(g, bh);
    const int n = k.Vb * nc;
    const int th = threads_for(n);
    dim3 grid(k.Vc / 2, nrhs);
    if (kprec == 0) {
        const size_t smem = 3 * (size_t)n * sizeof(cx<double>) + 3 * 32 * sizeof(double);
        cudaError_t e = cudaFuncSetAttribute(csap_half_kernel<double, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        (note_launch(), csap_half_kernel<double, false><<<grid, th, smem, st>>>(k, nc, colour, nmr, x_mode, B, b, x));
    } else {
        const size_t smem = 3 * (size_t)n * sizeof(cx<float>) + 3 * 32 * sizeof(float);
        auto fn = kprec == 2 ? csap_half_kernel<float, true> : csap_half_kernel<float, false>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        (note_launch(), fn<<<grid, th, smem, st>>>(k, nc, colour, nmr, x_mode, B, b, x));
    }
    return cudaGetLastError();
}
