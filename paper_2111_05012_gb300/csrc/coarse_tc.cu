// Multi-right-hand-side coarse stencil on the 5th-generation tensor cores:
// y_r(X) = sum_d B_d(X) x_r(X + d) for up to 16 right-hand sides r at once,
// with bfloat16 operands and FP32 accumulation in tensor memory (tcgen05).
//
// Per coarse site X the stencil is one dense complex contraction of the
// Nc x 9Nc row block [B_0(X) ... B_8(X)] with the 9Nc x n_rhs neighbour
// vectors.  It runs as one real GEMM
//   D (128 x 2P) = A (128 x 9Nc) . G^T,   G = [Re x; Im x] (2P rows),
// P = n_rhs padded to 8 or 16.  A holds the rows Re B(a) and Im B(a) of
// output a, ordered so that within every 32-row quarter lane l < 16 carries
// Re B(16w + l) and lane l + 16 carries Im B(16w + l): after tcgen05.ld each
// pair of lanes (l, l ^ 16) combines its rows with one warp shuffle,
//   y_re = Re B . Re x - Im B . Im x,   y_im = Im B . Re x + Re B . Im x.
// Rows 2Nc..127 of the M = 128 tile are never read back, so their part of
// the shared-memory span is not filled.
//
// Both operands arrive by bulk copies: A from a copy of the operator in the
// 8 x 8 core-matrix operand layout (K-major, no swizzle), one copy per site;
// G as nine copies (one per direction d) of the neighbours' vectors, packed
// once per call into the same layout with the k-groups outermost, so that
// the nine pieces concatenate along K.  Copies of the next site overlap the
// MMAs and the epilogue of the current one (two stages).  One thread issues
// the 9Nc/16 MMAs (M 128, N 2P, K 16) and commits them to an mbarrier.
//
// All waits are bounded: on a timeout the kernel records an error, waits
// (bounded) for its own bulk copies, releases its tensor memory and returns.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kTcThreads = 128;
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
    const __nv_bfloat16* xp;    // [V][nc/8][2P/8][8][8]: packed neighbour vectors
    float2* y;                  // [nrhs][V][nc]
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

// Shared-memory plan of one CTA (byte offsets).  An operator descriptor spans
// 16 row groups (M = 128) but only the first 2Nc/8 hold operator rows: the
// rest of the span may overlap the next buffer.
struct TcPlan {
    int a0, a1;   // operator buffers (a1 == a0: one buffer)
    int b0, b1;   // packed-vector buffers
    int bar;      // mbarriers
    int bytes;
};

// x [nrhs][V][nc] FP32 complex -> xp [V][nc/8][2P/8][8][8] bfloat16, row n = r (Re) / P + r (Im)
__global__ void tc_pack_kernel(int V, int nc, int nrhs, int P, const float2* __restrict__ x, __nv_bfloat16* xp) {
    const int NG = 2 * P / 8;
    const size_t per = (size_t)nc * 2 * P;
    const size_t n = (size_t)V * nc * P;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % nc);
        const size_t t = i / nc;
        const int Y = (int)(t % V), r = (int)(t / V);
        const float2 v = r < nrhs ? x[((size_t)r * V + Y) * nc + k] : make_float2(0.f, 0.f);
        __nv_bfloat16* o = xp + Y * per;
        const int re = r, im = P + r;
        o[((size_t)(k >> 3) * NG + (re >> 3)) * 64 + (re & 7) * 8 + (k & 7)] = __float2bfloat16(v.x);
        o[((size_t)(k >> 3) * NG + (im >> 3)) * 64 + (im & 7) * 8 + (k & 7)] = __float2bfloat16(v.y);
    }
}

template <int NP>   // NP = 2P accumulator columns (16 or 32)
__global__ void __launch_bounds__(kTcThreads, 1) coarse_tc_kernel(TcArgs a, TcPlan pl) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr int P = NP / 2, NG = NP / 8;
    const int nc = a.nc, K = 9 * nc, kg = K / 8;
    const unsigned a_bytes = (unsigned)(2 * nc) * K * 2;        // operator rows of one site
    const unsigned x_site = (unsigned)nc * NP * 2;              // packed vectors of one site
    unsigned char* Ab[2] = {smem_raw + pl.a0, smem_raw + pl.a1};
    unsigned char* Bb[2] = {smem_raw + pl.b0, smem_raw + pl.b1};
    const bool dblA = pl.a1 != pl.a0;
    uint64_t* barA = reinterpret_cast<uint64_t*>(smem_raw + pl.bar);   // [2]
    uint64_t* barB = barA + 2;                                           // [2]
    uint64_t* barM = barA + 4;
    uint32_t* slot = reinterpret_cast<uint32_t*>(barA + 5);
    int* fail = reinterpret_cast<int*>(slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nq = 2 * nc / 32;   // quarters of the accumulator holding operator rows

    if (tid == 0) {
        for (int i = 0; i < 5; ++i) mb_init(&barA[i], 1);
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
    const uint32_t a_lbo = 128, a_sbo = (uint32_t)kg * 128;   // A: [m group][k group][8][8]
    const uint32_t b_lbo = NG * 128, b_sbo = 128;             // G: [k group][n group][8][8]
    unsigned phA[2] = {0, 0}, phB[2] = {0, 0}, phM = 0;
    bool pendA[2] = {false, false}, pendB[2] = {false, false};   // thread 0 only
    auto issueA = [&](int X, int s) {
        mb_expect_tx(&barA[s], a_bytes);
        bulk_load(Ab[s], a.img + (size_t)X * (2 * nc) * K, a_bytes, &barA[s]);
        pendA[s] = true;
    };
    auto issueB = [&](int X, int s) {
        mb_expect_tx(&barB[s], 9 * x_site);
        for (int d = 0; d < 9; ++d)
            bulk_load(Bb[s] + d * x_site, a.xp + (size_t)tc_nbr(a, X, d) * (x_site / 2), x_site, &barB[s]);
        pendB[s] = true;
    };
    if (tid == 0 && (int)blockIdx.x < a.V) {
        issueA(blockIdx.x, 0);
        issueB(blockIdx.x, 0);
    }
    int it = 0;
    for (int X = blockIdx.x; X < a.V; X += gridDim.x, ++it) {
        const int sB = it & 1, sA = dblA ? (it & 1) : 0;
        const int Xn = X + gridDim.x;
        if (tid == 0) {
            // the other stage's buffers were last read by the previous site's MMAs, which completed
            if (Xn < a.V) {
                issueB(Xn, sB ^ 1);
                if (dblA) issueA(Xn, sA ^ 1);
            }
            if (mb_wait(&barA[sA], phA[sA]) && mb_wait(&barB[sB], phB[sB])) {
                pendA[sA] = pendB[sB] = false;
                phA[sA] ^= 1;
                phB[sB] ^= 1;
                tc_after();
                const uint32_t a0 = su32(Ab[sA]), b0 = su32(Bb[sB]);
                for (int q = 0; q < K / 16; ++q)
                    mma_bf16(tmem, smem_desc(a0 + q * 256, a_lbo, a_sbo), smem_desc(b0 + q * 2 * NG * 128, b_lbo, b_sbo),
                             idesc, q > 0 ? 1u : 0u);
                mma_commit(barM);
            } else {
                *fail = 1;
            }
        }
        __syncthreads();
        if (*fail) break;
        if (!mb_wait(barM, phM)) atomicExch(fail, 2);
        phM ^= 1;
        __syncthreads();
        if (*fail) break;
        tc_after();
        if (!dblA && tid == 0 && Xn < a.V) issueA(Xn, 0);   // the single operator buffer is free again
        if (warp < nq) {
            uint32_t v[NP];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
            if constexpr (NP == 32) tm_ld32(taddr, v);
            else tm_ld16(taddr, v);
            const int aa = warp * 16 + (lane & 15);
            const bool im = lane >= 16;
#pragma unroll
            for (int r = 0; r < P; ++r) {
                // Re row: y_re = ReB.Re x - ImB.Im x; Im row: y_im = ImB.Re x + ReB.Im x
                const float pv = __shfl_xor_sync(0xffffffffu, __uint_as_float(v[P + r]), 16);
                float val = im ? __uint_as_float(v[r]) + pv : __uint_as_float(v[r]) - pv;
                if (r < a.nrhs) {
                    const size_t o = ((size_t)r * a.V + X) * nc + aa;
                    float* yo = reinterpret_cast<float*>(a.y + o) + (im ? 1 : 0);
                    if (a.b) val = reinterpret_cast<const float*>(a.b + o)[im ? 1 : 0] - val;
                    *yo = val;
                }
            }
        }
        tc_before();
        __syncthreads();
        tc_after();
    }
    if (*fail && tid == 0) {
        // drain our own bulk copies before the shared memory goes away
        for (int s2 = 0; s2 < 2; ++s2) {
            if (pendA[s2]) mb_wait(&barA[s2], phA[s2]);
            if (pendB[s2]) mb_wait(&barB[s2], phB[s2]);
        }
        // a timed-out wait for the MMAs (fail 2) left them possibly still writing the
        // accumulator: wait for their commit once more (phM was flipped after the failed
        // wait); if that also gives up, the accumulator is not released (fail 3)
        if (*fail == 2 && !mb_wait(barM, phM ^ 1)) *fail = 3;
        atomicExch(a.err, 1);
    }
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0 && *fail != 3) tm_dealloc(tmem, 32);
}

// operator image: row m = 32 w + l holds Re (l < 16) or Im (l >= 16) of
// B[X][16 w + l % 16][d][col], column k = d * nc + col
__global__ void tc_image_kernel(int V, int nc, const float2* __restrict__ B, __nv_bfloat16* img) {
    const int K = 9 * nc, kg = K / 8;
    const size_t per = (size_t)2 * nc * K;
    const size_t n = (size_t)V * per;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t X = i / per;
        const int e = (int)(i - X * per);
        const int m = e / K, k = e - m * K;
        const int row = (m >> 5) * 16 + (m & 15);
        const float2 v = B[((size_t)X * nc + row) * K + k];   // [X][row][d][col] = [X][row][k]
        img[X * per + core_off(m, k, kg)] = __float2bfloat16((m & 16) ? v.y : v.x);
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

size_t coarse_tc_pack_bytes(int V, int nc) { return (size_t)V * nc * 32 * 2; }

cudaError_t launch_coarse_apply_tc(const GeomH& g, int nc, const void* img, const void* x, void* y, const void* b,
                                   int nrhs, void* xpack, int* err, cudaStream_t st) {
    if (!coarse_tc_supported(nc) || nrhs < 1 || nrhs > 16) return cudaErrorInvalidValue;
    TcArgs a;
    for (int i = 0; i < 4; ++i) a.L[i] = g.L[i];
    a.V = g.V;
    a.nc = nc;
    a.nrhs = nrhs;
    a.P = nrhs <= 8 ? 8 : 16;
    a.img = (const __nv_bfloat16*)img;
    a.xp = (const __nv_bfloat16*)xpack;
    a.y = (float2*)y;
    a.b = (const float2*)b;
    a.err = err;
    const int K = 9 * nc, kg = K / 8, NP = 2 * a.P;
    const int a_data = 2 * nc * K * 2, a_span = 16 * kg * 128, b_bytes = K * NP * 2;
    const int kMax = 227 * 1024;
    auto plan = [&](bool dbl) {
        TcPlan p;
        p.a0 = 0;
        p.a1 = dbl ? a_data : 0;
        p.b0 = p.a1 + a_data;
        p.b1 = p.b0 + b_bytes;
        p.bar = p.b1 + b_bytes;
        const int end = p.bar + 5 * 8 + 8;
        const int span = p.a1 + a_span;   // reach of the last operator descriptor
        p.bytes = ((end > span ? end : span) + 127) / 128 * 128;
        return p;
    };
    TcPlan pl = plan(true);
    if (pl.bytes > kMax) pl = plan(false);
    if (pl.bytes > kMax) return cudaErrorInvalidValue;
    (note_launch(), tc_pack_kernel<<<tc_sms() * 8, 256, 0, st>>>(g.V, nc, nrhs, a.P, (const float2*)x,
                                                                 (__nv_bfloat16*)xpack));
    const void* fn = NP == 32 ? (const void*)coarse_tc_kernel<32> : (const void*)coarse_tc_kernel<16>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.bytes);
    if (e != cudaSuccess) return e;
    const int grid = g.V < tc_sms() ? g.V : tc_sms();
    void* params[] = {&a, &pl};
    note_launch();
    return cudaLaunchKernel(fn, dim3(grid), dim3(kTcThreads), params, pl.bytes, st);
}
