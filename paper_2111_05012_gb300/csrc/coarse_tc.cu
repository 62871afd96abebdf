// Multi-right-hand-side coarse stencil on the 5th-generation tensor cores:
// y_r(X) = sum_d B_d(X) x_r(X + d) for up to 16 right-hand sides r at once,
// with bfloat16 operands and FP32 accumulation in tensor memory (tcgen05).
//
// Per coarse site X the stencil is one dense complex contraction of the
// Nc x 9Nc row block [B_0(X) ... B_8(X)] with the 9Nc x n_rhs gathered
// neighbour vectors.  It runs as one real GEMM
//   D (128 x 2P) = A (128 x 9Nc) . G^T,   A = [Re B; Im B] (rows 2Nc..127 zero),
//   G = [Re x; Im x] (2P rows, P = n_rhs padded to 8 or 16),
// after which y_re = D[a][r] - D[Nc+a][P+r] and y_im = D[Nc+a][r] + D[a][P+r].
// A is streamed from a copy of the operator stored in the tensor-core
// operand layout (8 x 8 core matrices, K-major, no swizzle) by one bulk copy
// per site; G is gathered by the CTA into the same layout; one thread issues
// the 9Nc/16 MMAs (M 128, N 2P, K 16) and commits them to an mbarrier; four
// warps read the accumulator rows back with tcgen05.ld.
//
// All waits are bounded: on a timeout the kernel records an error, waits
// (bounded) for its own bulk copy, releases its tensor memory and returns.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kTcThreads = 256;
constexpr long long kTcSpin = 20000000;

DEV uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
DEV void mb_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
DEV void mb_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
DEV void mb_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
DEV void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}
DEV bool mb_try(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
DEV bool mb_wait(uint64_t* bar, unsigned parity) {
    for (long long i = 0; i < kTcSpin; ++i)
        if (mb_try(bar, parity)) return true;
    return false;
}

// ---- tensor memory and tcgen05 (inline PTX) ----
DEV void tm_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(ncols)
                 : "memory");
}
DEV void tm_relinquish() { asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory"); }
DEV void tm_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
DEV void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
DEV void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
DEV void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// D (tmem) (+)= A (smem desc) . B (smem desc)^T, bf16 x bf16 -> f32
DEV void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
DEV void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
// 32 lanes x 32 columns (one row of 32 FP32 per thread) / 16 columns
DEV void tm_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
DEV void tm_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// shared-memory matrix descriptor: K-major, no swizzle; lbo = bytes between
// core matrices adjacent in K, sbo = bytes between core matrices adjacent in M/N
DEV uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of this architecture
    return d;                  // base offset 0, layout: no swizzle
}
// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, M x N
HD uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// element offset of (row, k) in an operand tile stored as [row/8][k/8][8][8]
HD size_t core_off(int row, int k, int kg) { return ((size_t)(row >> 3) * kg + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7); }

struct TcArgs {
    int L[4];
    int V, nc, nrhs, P;   // P: right-hand sides padded to 8 or 16
    const __nv_bfloat16* img;   // [V][2nc rows][9nc] in core-matrix order
    const float2* x;            // [nrhs][V][nc]
    float2* y;
    const float2* b;            // residual form y = b - D x when non-null
    int* err;
};

DEV int tc_nbr(const TcArgs& a, int X, int d) {
    if (d == 0) return X;
    int c[4];
    int t = X;
    c[0] = t % a.L[0];
    t /= a.L[0];
    c[1] = t % a.L[1];
    t /= a.L[1];
    c[2] = t % a.L[2];
    c[3] = t / a.L[2];
    const int mu = (d - 1) & 3;
    c[mu] = d <= 4 ? (c[mu] + 1 == a.L[mu] ? 0 : c[mu] + 1) : (c[mu] == 0 ? a.L[mu] - 1 : c[mu] - 1);
    return c[0] + a.L[0] * (c[1] + a.L[1] * (c[2] + a.L[2] * c[3]));
}

// Shared-memory plan of one CTA (byte offsets; see coarse_tc_plan).  A
// descriptor always spans 16 row groups (M = 128), but only the first 2Nc/8
// hold operator rows: the rest of the span may overlap the next buffer, and
// the accumulator rows it produces (2Nc..127) are never read.
struct TcPlan {
    int a0, a1;        // operator buffers (a1 == a0: single buffer)
    int bsm, dsm, bar; // gathered vectors, accumulator staging, mbarriers
    int bytes;         // dynamic shared memory to request
};

template <int NP>   // NP = 2P accumulator columns (16 or 32)
__global__ void __launch_bounds__(kTcThreads, 1) coarse_tc_kernel(TcArgs a, TcPlan pl) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int nc = a.nc, K = 9 * nc, kg = K / 8, pairs = nc / 2;
    const unsigned a_bytes = (unsigned)(2 * nc) * K * 2;   // operator rows of one site
    unsigned char* Abuf[2] = {smem_raw + pl.a0, smem_raw + pl.a1};
    const bool dbl = pl.a1 != pl.a0;
    __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(smem_raw + pl.bsm);
    float* Ds = reinterpret_cast<float*>(smem_raw + pl.dsm);   // [128][NP]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + pl.bar);   // [0], [1] operator copies, [2] MMA
    uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 3);
    int* fail = reinterpret_cast<int*>(slot + 1);
    int* nbr = fail + 1;   // [9] neighbour sites of the current coarse site
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        mb_init(&bars[0], 1);
        mb_init(&bars[1], 1);
        mb_init(&bars[2], 1);
        mb_fence_init();
        *fail = 0;
    }
    if (warp == 0) {
        tm_alloc(slot, 32);
        tm_relinquish();
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *slot;
    const uint32_t idesc = idesc_bf16(128, NP);
    const uint32_t lbo = 128, sbo = (uint32_t)kg * 128;
    unsigned ph[2] = {0, 0}, ph_m = 0;
    bool pend[2] = {false, false};   // meaningful in thread 0 only
    auto issue = [&](int X, int b) {
        mb_expect_tx(&bars[b], a_bytes);
        bulk_load(Abuf[b], a.img + (size_t)X * (2 * nc) * K, a_bytes, &bars[b]);
        pend[b] = true;
    };
    if (tid == 0 && blockIdx.x < a.V) issue(blockIdx.x, 0);

    int it = 0;
    for (int X = blockIdx.x; X < a.V; X += gridDim.x, ++it) {
        const int sel = dbl ? (it & 1) : 0;
        const int Xn = X + gridDim.x;
        if (dbl && tid == 0 && Xn < a.V) issue(Xn, sel ^ 1);   // its buffer was last read by the previous MMA
        if (tid < 9) nbr[tid] = tc_nbr(a, X, tid);
        __syncthreads();
        // gather G: row r = Re x_r, row P + r = Im x_r, column k = d * nc + b, two complex per load
        const int items = a.P * 9 * pairs;
        for (int base = tid; base < items; base += kTcThreads * 4) {
            float4 v[4];
            int rr[4], kk[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = base + u * kTcThreads;
                rr[u] = -1;
                if (idx < items) {
                    const int r = idx / (9 * pairs), rem = idx - r * 9 * pairs;
                    const int d = rem / pairs, c2 = rem - d * pairs;
                    rr[u] = r;
                    kk[u] = d * nc + 2 * c2;
                    v[u] = r < a.nrhs ? __ldg(reinterpret_cast<const float4*>(a.x) +
                                              ((size_t)r * a.V + nbr[d]) * pairs + c2)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (rr[u] < 0) continue;
                *reinterpret_cast<__nv_bfloat162*>(Bs + core_off(rr[u], kk[u], kg)) = __floats2bfloat162_rn(v[u].x, v[u].z);
                *reinterpret_cast<__nv_bfloat162*>(Bs + core_off(a.P + rr[u], kk[u], kg)) =
                    __floats2bfloat162_rn(v[u].y, v[u].w);
            }
        }
        proxy_fence();
        __syncthreads();
        if (tid == 0) {
            if (mb_wait(&bars[sel], ph[sel])) {
                pend[sel] = false;
                ph[sel] ^= 1;
                tc_after();
                const uint32_t a0 = su32(Abuf[sel]), b0 = su32(Bs);
                for (int q = 0; q < K / 16; ++q)
                    mma_bf16(tmem, smem_desc(a0 + q * 256, lbo, sbo), smem_desc(b0 + q * 256, lbo, sbo), idesc,
                             q > 0 ? 1u : 0u);
                mma_commit(&bars[2]);
            } else {
                *fail = 1;
            }
        }
        __syncthreads();
        if (*fail) break;
        if (!mb_wait(&bars[2], ph_m)) atomicExch(fail, 2);
        ph_m ^= 1;
        __syncthreads();
        if (*fail) break;
        tc_after();
        // the operator buffer is free again: fetch the next site's rows during the epilogue
        if (!dbl && tid == 0 && Xn < a.V) issue(Xn, 0);
        if (warp < 4) {
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
            const int row = warp * 32 + lane;
            if (NP == 32) {
                uint32_t r[32];
                tm_ld32(taddr, r);
#pragma unroll
                for (int c = 0; c < 32; ++c) Ds[row * NP + c] = __uint_as_float(r[c]);
            } else {
                uint32_t r[16];
                tm_ld16(taddr, r);
#pragma unroll
                for (int c = 0; c < 16; ++c) Ds[row * NP + c] = __uint_as_float(r[c]);
            }
        }
        tc_before();
        __syncthreads();
        for (int idx = tid; idx < nc * a.nrhs; idx += kTcThreads) {
            const int r = idx / nc, aa = idx - r * nc;
            float yr = Ds[aa * NP + r] - Ds[(nc + aa) * NP + a.P + r];
            float yi = Ds[(nc + aa) * NP + r] + Ds[aa * NP + a.P + r];
            const size_t o = ((size_t)r * a.V + X) * nc + aa;
            if (a.b) {
                const float2 bv = a.b[o];
                yr = bv.x - yr;
                yi = bv.y - yi;
            }
            a.y[o] = make_float2(yr, yi);
        }
        __syncthreads();
    }
    if (*fail) {
        if (tid == 0) {
            // drain our own bulk copies before the shared memory goes away
            for (int b = 0; b < 2; ++b)
                if (pend[b]) mb_wait(&bars[b], ph[b]);
            atomicExch(a.err, 1);
        }
    }
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0) tm_dealloc(tmem, 32);
}

// operator image: row m < nc: Re B[X][m][d][col], m >= nc: Im B[X][m - nc][d][col], k = d * nc + col
__global__ void tc_image_kernel(int V, int nc, const float2* __restrict__ B, __nv_bfloat16* img) {
    const int K = 9 * nc, kg = K / 8;
    const size_t per = (size_t)2 * nc * K;
    const size_t n = (size_t)V * per;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t X = i / per;
        const int e = (int)(i - X * per);
        const int m = e / K, k = e - m * K;
        const int row = m < nc ? m : m - nc;
        const float2 v = B[((size_t)X * nc + row) * K + k];   // [X][row][d][col] = [X][row][k]
        img[X * per + core_off(m, k, kg)] = __float2bfloat16(m < nc ? v.x : v.y);
    }
}

int tc_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

bool coarse_tc_supported(int nc) { return nc > 0 && nc % 16 == 0 && nc <= 64; }
size_t coarse_tc_image_bytes(int V, int nc) { return (size_t)V * 2 * nc * 9 * nc * 2; }

cudaError_t launch_coarse_tc_image(int V, int nc, const void* B32, void* img, cudaStream_t st) {
    if (!coarse_tc_supported(nc)) return cudaErrorInvalidValue;
    (note_launch(), tc_image_kernel<<<tc_sms() * 8, 256, 0, st>>>(V, nc, (const float2*)B32, (__nv_bfloat16*)img));
    return cudaGetLastError();
}

cudaError_t launch_coarse_apply_tc(const GeomH& g, int nc, const void* img, const void* x, void* y, const void* b,
                                   int nrhs, int* err, cudaStream_t st) {
    if (!coarse_tc_supported(nc) || nrhs < 1 || nrhs > 16) return cudaErrorInvalidValue;
    TcArgs a;
    for (int i = 0; i < 4; ++i) a.L[i] = g.L[i];
    a.V = g.V;
    a.nc = nc;
    a.nrhs = nrhs;
    a.P = nrhs <= 8 ? 8 : 16;
    a.img = (const __nv_bfloat16*)img;
    a.x = (const float2*)x;
    a.y = (float2*)y;
    a.b = (const float2*)b;
    a.err = err;
    const int K = 9 * nc, kg = K / 8, NP = 2 * a.P;
    const int a_data = 2 * nc * K * 2, a_span = 16 * kg * 128;
    const int b_bytes = (NP / 8) * kg * 128, d_bytes = 128 * NP * 4, tail = 3 * 8 + 4 + 4 + 9 * 4;
    const int kMax = 227 * 1024;
    auto plan = [&](bool dbl) {
        TcPlan p;
        p.a0 = 0;
        p.a1 = dbl ? a_data : 0;
        p.bsm = (dbl ? 2 * a_data : a_data);
        p.dsm = p.bsm + b_bytes;
        p.bar = p.dsm + d_bytes;
        const int end = p.bar + tail;
        const int span = p.a1 + a_span;   // the last operator descriptor's reach
        p.bytes = ((end > span ? end : span) + 127) / 128 * 128;
        return p;
    };
    TcPlan pl = plan(true);
    if (pl.bytes > kMax) pl = plan(false);
    if (pl.bytes > kMax) return cudaErrorInvalidValue;
    const void* fn = NP == 32 ? (const void*)coarse_tc_kernel<32> : (const void*)coarse_tc_kernel<16>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.bytes);
    if (e != cudaSuccess) return e;
    const int grid = g.V < tc_sms() ? g.V : tc_sms();
    void* params[] = {&a, &pl};
    note_launch();
    return cudaLaunchKernel(fn, dim3(grid), dim3(kTcThreads), params, pl.bytes, st);
}
