// Coarse-lattice kernels: the 9-point block stencil y(X) = sum_d B[X][d] x(X+d)
// of the Galerkin operator (Eq. 7) and precision conversion of flat complex
// arrays.  Internal stencil layout [X][row][d][col] (complex, row-major) so
// that one output row reads one contiguous run of 9 * Nc entries.
#include "common.cuh"
#include "kernels.h"

namespace {

template <typename TC> struct C2T;
template <> struct C2T<double> { using V = double2; };
template <> struct C2T<float> { using V = float2; };

template <typename TC> DEV cx<TC> ldc(const void* p, size_t i) {
    typename C2T<TC>::V t = __ldg((const typename C2T<TC>::V*)p + i);
    return {t.x, t.y};
}
template <typename TC> DEV void stc(void* p, size_t i, cx<TC> v) {
    ((typename C2T<TC>::V*)p)[i] = {v.re, v.im};
}

struct CGeom {
    int L[4];
    int V;
};
DEV int cneighbour(const CGeom& g, int X, int d, int c[4]) {
    // d = 0 self, 1+mu forward, 5+mu backward (periodic; boundary phases live in B)
    if (d == 0) return X;
    int mu = (d - 1) % 4, dir = d <= 4 ? 1 : -1;
    int cc[4] = {c[0], c[1], c[2], c[3]};
    cc[mu] = (cc[mu] + dir + g.L[mu]) % g.L[mu];
    return cc[0] + g.L[0] * (cc[1] + g.L[1] * (cc[2] + g.L[2] * cc[3]));
}

// One CTA per coarse site; the 9 neighbour vectors are gathered into shared
// memory, each warp then produces output rows (lanes stride over 9*Nc).
// sap: hops that cross a block boundary of size sb are dropped (D_SAP).
// operator entry i in the storage ST: 0 the arithmetic precision TC, 1 bfloat16
// (TC = float), 2 FP32 widened to TC = double (the entries are FP32-exact)
template <typename TC, int ST> DEV cx<TC> ldb(const void* B, size_t i) { return ldc<TC>(B, i); }
template <> DEV cx<float> ldb<float, 1>(const void* B, size_t i) {
    float2 f = __bfloat1622float2(__ldg((const __nv_bfloat162*)B + i));
    return {f.x, f.y};
}
template <> DEV cx<double> ldb<double, 2>(const void* B, size_t i) {
    float2 f = __ldg((const float2*)B + i);
    return {(double)f.x, (double)f.y};
}

template <typename TC, bool RESID, int BF = 0>
__global__ void coarse_apply_kernel(CGeom g, int nc, int sap, int4 sb, const void* __restrict__ B,
                                    const void* __restrict__ in, void* out, const void* __restrict__ b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<TC>* xin = reinterpret_cast<cx<TC>*>(smem_raw);   // [9][nc]
    const int r = blockIdx.y;
    const size_t off = (size_t)r * g.V * nc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int sbv[4] = {sb.x, sb.y, sb.z, sb.w};
    for (int X = blockIdx.x; X < g.V; X += gridDim.x) {
        int c[4];
        c[0] = X % g.L[0];
        int t = X / g.L[0];
        c[1] = t % g.L[1];
        t /= g.L[1];
        c[2] = t % g.L[2];
        c[3] = t / g.L[2];
        for (int idx = threadIdx.x; idx < 9 * nc; idx += blockDim.x) {
            int d = idx / nc, col = idx % nc;
            bool keep = true;
            if (sap && d > 0) {
                int mu = (d - 1) % 4;
                int lc = c[mu] % sbv[mu];
                keep = d <= 4 ? (lc != sbv[mu] - 1) : (lc != 0);
            }
            cx<TC> v = czero<TC>();
            if (keep) v = ldc<TC>(in, off + (size_t)cneighbour(g, X, d, c) * nc + col);
            xin[idx] = v;
        }
        __syncthreads();
        for (int row = warp; row < nc; row += nw) {
            const size_t base = ((size_t)X * nc + row) * 9 * nc;
            cx<TC> acc = czero<TC>();
            for (int j = lane; j < 9 * nc; j += 32) cfma(acc, ldb<TC, BF>(B, base + j), xin[j]);
            acc.re = warp_sum(acc.re);
            acc.im = warp_sum(acc.im);
            if (lane == 0) {
                if (RESID) acc = ldc<TC>(b, off + (size_t)X * nc + row) - acc;
                stc<TC>(out, off + (size_t)X * nc + row, acc);
            }
        }
        __syncthreads();
    }
}

template <typename TC>
__global__ void coarse_export_kernel(int Vc, int nc, const void* B, double* out) {
    const size_t n = (size_t)Vc * 9 * nc * nc;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        // out index [X][d][row][col]
        size_t col = i % nc, rest = i / nc;
        size_t row = rest % nc;
        rest /= nc;
        size_t d = rest % 9, X = rest / 9;
        cx<TC> v = ldc<TC>(B, ((X * nc + row) * 9 + d) * nc + col);
        out[2 * i] = (double)v.re;
        out[2 * i + 1] = (double)v.im;
    }
}

template <typename TI, typename TO>
__global__ void convert_flat_kernel(const void* in, void* out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        stc<TO>(out, i, ccast<TO>(ldc<TI>(in, i)));
}

__global__ void to_bf16_kernel(const float2* __restrict__ in, __nv_bfloat162* out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __float22bfloat162_rn(in[i]);
}

int nsm() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

}  // namespace

cudaError_t launch_coarse_apply(int cprec, const GeomH& gh, int nc, const BlockH* sb, const void* B, const void* in,
                                void* out, const void* b, int nrhs, cudaStream_t st) {
    CGeom g;
    for (int i = 0; i < 4; ++i) g.L[i] = gh.L[i];
    g.V = gh.V;
    int4 blk = sb ? make_int4(sb->b[0], sb->b[1], sb->b[2], sb->b[3]) : make_int4(1, 1, 1, 1);
    int sap = sb != nullptr;
    dim3 grid(g.V < nsm() * 8 ? g.V : nsm() * 8, nrhs);
    int th = 256;
    if (cprec == 0 || cprec == 3) {   // FP64 vectors; operator FP64 (0) or FP32-exact stored in FP32 (3)
        size_t smem = (size_t)9 * nc * sizeof(cx<double>);
        if (cprec == 3) {
            if (b) (note_launch(), coarse_apply_kernel<double, true, 2><<<grid, th, smem, st>>>(g, nc, sap, blk, B, in, out, b));
            else (note_launch(), coarse_apply_kernel<double, false, 2><<<grid, th, smem, st>>>(g, nc, sap, blk, B, in, out, b));
        } else {
            if (b) (note_launch(), coarse_apply_kernel<double, true><<<grid, th, smem, st>>>(g, nc, sap, blk, B, in, out, b));
            else (note_launch(), coarse_apply_kernel<double, false><<<grid, th, smem, st>>>(g, nc, sap, blk, B, in, out, b));
        }
    } else {
        size_t smem = (size_t)9 * nc * sizeof(cx<float>);
        if (cprec == 2) {   // FP32 vectors, bfloat16 operator
            if (b) (note_launch(), coarse_apply_kernel<float, true, 1><<<grid, th, smem, st>>>(g, nc, sap, blk, B, in, out, b));
            else (note_launch(), coarse_apply_kernel<float, false, 1><<<grid, th, smem, st>>>(g, nc, sap, blk, B, in, out, b));
        } else {
            if (b) (note_launch(), coarse_apply_kernel<float, true><<<grid, th, smem, st>>>(g, nc, sap, blk, B, in, out, b));
            else (note_launch(), coarse_apply_kernel<float, false><<<grid, th, smem, st>>>(g, nc, sap, blk, B, in, out, b));
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_coarse_op_export(int cprec, int Vc, int nc, const void* B, double* out, cudaStream_t st) {
    int grid = nsm() * 8;
    if (cprec == 0) (note_launch(), coarse_export_kernel<double><<<grid, 256, 0, st>>>(Vc, nc, B, out));
    else (note_launch(), coarse_export_kernel<float><<<grid, 256, 0, st>>>(Vc, nc, B, out));
    return cudaGetLastError();
}

cudaError_t launch_convert_flat(int pi, int po, const void* in, void* out, size_t n, cudaStream_t st) {
    int grid = nsm() * 8;
    if (pi == 0 && po == 1) (note_launch(), convert_flat_kernel<double, float><<<grid, 256, 0, st>>>(in, out, n));
    else if (pi == 1 && po == 0) (note_launch(), convert_flat_kernel<float, double><<<grid, 256, 0, st>>>(in, out, n));
    else if (pi == 0) (note_launch(), convert_flat_kernel<double, double><<<grid, 256, 0, st>>>(in, out, n));
    else (note_launch(), convert_flat_kernel<float, float><<<grid, 256, 0, st>>>(in, out, n));
    return cudaGetLastError();
}

cudaError_t launch_complex_to_bf16(const void* in, void* out, size_t n, cudaStream_t st) {
    (note_launch(), to_bf16_kernel<<<nsm() * 8, 256, 0, st>>>((const float2*)in, (__nv_bfloat162*)out, n));
    return cudaGetLastError();
}
