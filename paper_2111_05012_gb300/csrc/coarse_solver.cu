// Persistent coarse-grid solver: BiCGStab(l) (Sleijpen-Fokkema) for the
// coarse system D_c x = b of step (1b) in Sec. 3, run to a loose relative
// tolerance entirely on the device in ONE cooperative launch.
//
// Every CTA owns a contiguous range of rows of the coarse system; a warp
// computes one row of the 9-point stencil at a time and all elementwise
// vector updates of a row are done by the CTA that owns it, so vector
// dependencies only cross CTAs at the stencil's neighbour reads.  Grid-wide
// reductions write one FP64 partial per CTA; after a grid barrier every CTA
// sums the partials in the same fixed order, so all CTAs hold bit-identical
// scalars and take identical branches.  The minimal-residual part uses the
// Gram matrix of R_0..R_l (one reduction) instead of sequential projections.
//
// The stencil streams the CTA's contiguous slice of the coarse operator
// through a 3-stage shared-memory ring filled by bulk asynchronous copies
// (cp.async.bulk, completion counted on mbarriers); the neighbour vector
// segments a chunk needs ride in the same ring slot, one bulk copy per
// (site, direction).
//
// Grid barriers and mbarrier waits spin with a bounded count; on timeout the
// kernel records AMG_TIMEOUT in the status word and every CTA returns.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxEll = 4;
constexpr int kMaxQ = (kMaxEll + 1) * (kMaxEll + 1) + 2;   // reduced quantities per barrier
constexpr long long kSpinLimit = 40000000;                    // ~ seconds of polling
constexpr int kStages = 3;                                    // bulk-copy ring depth
constexpr int kChunkBytes = 55296;                            // operator bytes per ring slot (16 FP32 rows, Nc 48)
constexpr int kMaxRowsPerWarp = 4;                            // rows of one chunk per warp (the launcher checks)

struct GridBar {
    unsigned count;
    unsigned gen;
    int err;
    int cycles;
};

template <typename TC> struct V2;
template <> struct V2<double> { using T = double2; };
template <> struct V2<float> { using T = float2; };

// vectors are written by other CTAs of the same grid: read them through L2
// (ld.global.cg), never from a possibly stale L1 line
template <typename TC> DEV cx<TC> ld(const void* p, size_t i) {
    typename V2<TC>::T t = __ldcg((const typename V2<TC>::T*)p + i);
    return {t.x, t.y};
}
template <typename TC> DEV cx<TC> ldg(const void* p, size_t i) {
    typename V2<TC>::T t = __ldg((const typename V2<TC>::T*)p + i);
    return {t.x, t.y};
}
template <typename TC> DEV void st(void* p, size_t i, cx<TC> v) { ((typename V2<TC>::T*)p)[i] = {v.re, v.im}; }

// ---- mbarrier / bulk copy (inline PTX) ----
DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
DEV void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
DEV void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
DEV void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
DEV void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
DEV bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false after kSpinLimit polls
DEV bool mbar_wait(uint64_t* bar, unsigned parity) {
    for (long long it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

struct Args {
    int L[4];
    int Vc, nc, ell, maxit;
    double tol;
    const void* B;
    const void* b;
    void* x;
    void* rt;
    void* R[kMaxEll + 1];
    void* U[kMaxEll + 1];
    double2* part;   // [kMaxQ][gridDim.x]
    GridBar* bar;
    int rows_per_chunk;   // rows of the operator per ring slot
    int row_bytes;        // 9 * nc * sizeof(complex)
    int sites_per_chunk;  // coarse sites a chunk can touch: (rows_per_chunk - 1) / nc + 2
    int xseg_bytes;       // nc * sizeof(complex): one neighbour vector segment
    int slot_bytes;       // bytes per ring slot (kChunkBytes)
};

// ring state of one CTA (identical in all its threads)
struct Ring {
    unsigned char* buf;   // kStages slots of chunk bytes
    uint64_t* full;       // kStages mbarriers
    unsigned next;        // global index of the next chunk to consume
};

DEV unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
DEV unsigned atom_add_acqrel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
DEV void st_relaxed(unsigned* p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
DEV void red_release(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// grid barrier (sense by generation counter, acquire/release atomics); the
// CTA's writes are published by __syncthreads + the releasing arrival.
// Returns false if it gave up (then the caller returns).
DEV bool grid_sync(GridBar* gb) {
    __shared__ int s_ok;
    // vectors written here are read by bulk copies (async proxy) after the barrier
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int* verr = &gb->err;
        const unsigned g = ld_acquire(&gb->gen);
        int ok = 1;
        if (atom_add_acqrel(&gb->count, 1u) == gridDim.x - 1) {
            st_relaxed(&gb->count, 0u);
            red_release(&gb->gen, 1u);
        } else {
            long long it = 0;
            while (ld_acquire(&gb->gen) == g) {
                if (*verr) {
                    ok = 0;
                    break;
                }
                if (++it > kSpinLimit) {
                    atomicExch(&gb->err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(20);
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// CTA-wide sum of nq complex values held per thread (accumulated in AT, the
// solver's precision); thread 0 writes the CTA partials in FP64, the grid
// barrier follows, then every CTA sums all partials in fixed order.  Results
// land in `out` (shared) for all threads.
template <int NQ, typename AT>
DEV bool grid_reduce(const Args& a, cx<AT> (&v)[NQ], int nq, cx<double>* red_sh, cx<double>* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < nq; ++q) {
        AT re = warp_sum(v[q].re), im = warp_sum(v[q].im);
        if (lane == 0) red_sh[q * kWarps + warp] = {(double)re, (double)im};
    }
    __syncthreads();
    if (threadIdx.x < nq) {
        cx<double> t = czero<double>();
        for (int w = 0; w < kWarps; ++w) t = t + red_sh[threadIdx.x * kWarps + w];
        a.part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = make_double2(t.re, t.im);
    }
    if (!grid_sync(a.bar)) return false;
    // one warp per quantity, lanes stride over the CTA partials (fixed order)
    for (int q = warp; q < nq; q += kWarps) {
        double re = 0, im = 0;
        // up to 8 partials per lane (grids of <= 256 CTAs), loaded before any is summed so
        // that the L2 round trips overlap; the order of the sum is fixed
        constexpr int kPer = 8;
        double2 t[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = lane + 32 * k;
            t[k] = i < (int)gridDim.x ? __ldcg(a.part + (size_t)q * gridDim.x + i) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            re += t[k].x;
            im += t[k].y;
        }
        for (int i = lane + 32 * kPer; i < (int)gridDim.x; i += 32) {
            double2 u = __ldcg(a.part + (size_t)q * gridDim.x + i);
            re += u.x;
            im += u.y;
        }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) out[q] = {re, im};
    }
    __syncthreads();
    return true;
}

// row range owned by this CTA
DEV void my_rows(int nrows, int& r0, int& r1) {
    int per = (nrows + gridDim.x - 1) / gridDim.x;
    r0 = blockIdx.x * per;
    r1 = min(nrows, r0 + per);
    if (r0 > nrows) r0 = nrows;
}

// y(row) = sum_{d,col} B[row][d][col] x(nbr(X, d))[col] for the rows of this CTA
// (one warp per row); returns per-thread partial <w, y> if w != nullptr.
DEV int coarse_neighbour(const Args& a, int X, int d) {
    if (d == 0) return X;
    int c[4];
    c[0] = X % a.L[0];
    int t = X / a.L[0];
    c[1] = t % a.L[1];
    t /= a.L[1];
    c[2] = t % a.L[2];
    c[3] = t / a.L[2];
    const int mu = (d - 1) & 3, dir = d <= 4 ? 1 : -1;
    c[mu] = (c[mu] + dir + a.L[mu]) % a.L[mu];
    return c[0] + a.L[0] * (c[1] + a.L[1] * (c[2] + a.L[2] * c[3]));
}

// issue, from warp 0, the bulk copies of chunk c of this call into its ring
// slot: the chunk's operator rows, and the nine neighbour segments (nc
// entries each) of every coarse site the chunk touches, laid out as segment
// (s * 9 + d) for site X0 + s and direction d.  All complete on the slot's
// mbarrier, so the vector gather is as asynchronous as the operator stream.
template <typename TC>
DEV void ring_issue(const Args& a, Ring& rg, unsigned gidx, int r0, int r1, int c, const void* xin, cx<TC>* xbuf,
                    int xcap) {
    const int lane = threadIdx.x & 31;
    const int rc0 = r0 + c * a.rows_per_chunk;
    const int rows = min(r1 - rc0, a.rows_per_chunk);
    const unsigned slot = gidx % kStages;
    const int X0 = rc0 / a.nc, ns = (rc0 + rows - 1) / a.nc - X0 + 1;
    const unsigned seg = (unsigned)a.xseg_bytes;
    if (lane == 0) {
        // the transaction count is raised before any copy of this phase can complete
        mbar_expect_tx(&rg.full[slot], (unsigned)rows * (unsigned)a.row_bytes + (unsigned)(ns * 9) * seg);
        bulk_g2s(rg.buf + (size_t)slot * kChunkBytes, (const unsigned char*)a.B + (size_t)rc0 * a.row_bytes,
                 (unsigned)rows * (unsigned)a.row_bytes, &rg.full[slot]);
    }
    __syncwarp();
    // the vector was written through the generic proxy before the grid barrier
    asm volatile("fence.proxy.async.global;" ::: "memory");
    cx<TC>* xs = xbuf + (size_t)slot * xcap;
    for (int j = lane; j < ns * 9; j += 32) {
        const int sl = j / 9, d = j - 9 * sl;
        bulk_g2s(xs + (size_t)j * a.nc, (const cx<TC>*)xin + (size_t)coarse_neighbour(a, X0 + sl, d) * a.nc, seg,
                 &rg.full[slot]);
    }
}

// operator entries in shared memory: complex in the solver precision, or
// bfloat16 pairs (BF16 storage, FP32 arithmetic)
template <typename TC, bool BF> struct OpElem;
template <typename TC> struct OpElem<TC, false> {
    static constexpr int bytes = (int)sizeof(cx<TC>);
    DEV static cx<TC> get(const unsigned char* row, int e) { return ((const cx<TC>*)row)[e]; }
};
template <> struct OpElem<float, true> {
    static constexpr int bytes = 4;
    DEV static cx<float> get(const unsigned char* row, int e) {
        float2 f = __bfloat1622float2(((const __nv_bfloat162*)row)[e]);
        return {f.x, f.y};
    }
};

// y(row) = sum_{d,col} B[row][d][col] x(nbr(X, d))[col] for the rows of this CTA:
// operator rows and the neighbour segments of their sites arrive by bulk copy
// through the ring (kStages chunks in flight), and one warp computes one row
// entirely from shared memory; returns the per-thread partial <w, y> in dotp.
// Returns false if a ring wait timed out.  xin must have been made visible to
// the async proxy (fence.proxy.async before the grid barrier that precedes).
template <typename TC, bool BF>
DEV bool stencil_rows(const Args& a, Ring& rg, cx<TC>* xbuf, const void* xin, void* yout, const void* w, int r0,
                      int r1, cx<TC>& dotp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nc = a.nc, K = 9 * nc;
    const int xcap = 9 * a.sites_per_chunk * nc;   // complex numbers per slot's segment buffer
    const int nch = (r1 - r0 + a.rows_per_chunk - 1) / a.rows_per_chunk;
    const unsigned base = rg.next;
    int issued = min(nch, kStages);
    if (warp == 0)
        for (int c = 0; c < issued; ++c) ring_issue<TC>(a, rg, base + c, r0, r1, c, xin, xbuf, xcap);
    bool ok = true;
    // every issued chunk is waited for (bounded), even after a failure, so no
    // bulk copy is left in flight when the CTA returns
    for (int c = 0; c < issued; ++c) {
        const unsigned gidx = base + c, slot = gidx % kStages;
        const int rc0 = r0 + c * a.rows_per_chunk, rc1 = min(r1, rc0 + a.rows_per_chunk);
        // w at this warp's rows of the chunk, loaded before the wait so that the
        // L2 round trip overlaps it (a chunk has at most kMaxRowsPerWarp rows per warp)
        cx<TC> wv[kMaxRowsPerWarp];
        if (w && lane == 0) {
#pragma unroll
            for (int k = 0; k < kMaxRowsPerWarp; ++k) {
                const int r = rc0 + warp + k * kWarps;
                wv[k] = r < rc1 ? ld<TC>(w, r) : czero<TC>();
            }
        }
        const bool got = mbar_wait(&rg.full[slot], (gidx / kStages) & 1);
        ok = __syncthreads_and(ok && got) != 0;   // CTA-uniform
        const unsigned char* sb = rg.buf + (size_t)slot * kChunkBytes;
        const cx<TC>* xs = xbuf + (size_t)slot * xcap;
        const int X0 = rc0 / nc;
#pragma unroll 1
        for (int k = 0; k < kMaxRowsPerWarp; ++k) {
            const int r = rc0 + warp + k * kWarps;
            if (!ok || r >= rc1) break;
            const unsigned char* brow = sb + (size_t)(r - rc0) * a.row_bytes;
            const cx<TC>* xrow = xs + (size_t)(r / nc - X0) * K;   // the nine segments of this row's site
            cx<TC> acc0 = czero<TC>(), acc1 = czero<TC>();
#pragma unroll 4
            for (int j = lane; j < K / 2; j += 32) {
                acc0 = acc0 + OpElem<TC, BF>::get(brow, 2 * j) * xrow[2 * j];
                acc1 = acc1 + OpElem<TC, BF>::get(brow, 2 * j + 1) * xrow[2 * j + 1];
            }
            cx<TC> acc = acc0 + acc1;
            acc.re = warp_sum(acc.re);
            acc.im = warp_sum(acc.im);
            if (lane == 0) {
                st<TC>(yout, r, acc);
                if (w) {
                    cx<TC> wr = wv[0];
#pragma unroll
                    for (int q = 1; q < kMaxRowsPerWarp; ++q)
                        if (k == q) wr = wv[q];
                    dotp = dotp + cmulc(wr, acc);
                }
            }
        }
        __syncthreads();   // slot free again
        if (ok && c + kStages < nch) {
            if (warp == 0) ring_issue<TC>(a, rg, base + c + kStages, r0, r1, c + kStages, xin, xbuf, xcap);
            ++issued;
        }
    }
    rg.next = base + issued;
    return ok;
}

template <typename TC, bool BF>
__global__ void __launch_bounds__(kThreads) coarse_bicgstab_kernel(Args a) {
    __shared__ cx<double> red_sh[kMaxQ * kWarps];
    __shared__ cx<double> res[kMaxQ];
    __shared__ __align__(8) uint64_t full[kStages];
    extern __shared__ __align__(128) unsigned char ring_buf[];
    Ring rg{ring_buf, full, 0u};
    cx<TC>* xbuf = (cx<TC>*)(ring_buf + (size_t)kStages * kChunkBytes);   // kStages x 9 * sites_per_chunk * nc
    if (threadIdx.x == 0) {
        for (int k = 0; k < kStages; ++k) mbar_init(&full[k], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const int ell = a.ell;
    const int n = a.Vc * a.nc;
    int r0, r1;
    my_rows(n, r0, r1);
    const int tid = threadIdx.x;
    // initial state: x = 0, R0 = b, rt = b, U0 = 0
    for (int i = r0 + tid; i < r1; i += kThreads) {
        cx<TC> bi = ld<TC>(a.b, i);
        st<TC>(a.x, i, czero<TC>());
        st<TC>(a.R[0], i, bi);
        st<TC>(a.rt, i, bi);
        st<TC>(a.U[0], i, czero<TC>());
    }
    // BiCG scalars in the solver's precision: identical in every thread
    using SC = TC;
    // n / d with both scaled by max(|d.re|, |d.im|) first: the BiCG scalars are
    // squares of the residual scale, so |d|^2 would underflow (FP32) for the
    // small right-hand sides a non-normalising outer solver hands down
    auto cdiv = [](cx<SC> n, cx<SC> d) -> cx<SC> {
        const SC m = fmax(fabs(d.re), fabs(d.im));
        const SC sc = m > SC(0) ? SC(1) / m : SC(1);
        const cx<SC> ds = {d.re * sc, d.im * sc}, ns = {n.re * sc, n.im * sc};
        const SC inv = SC(1) / norm2(ds);
        return {(ns.re * ds.re + ns.im * ds.im) * inv, (ns.im * ds.re - ns.re * ds.im) * inv};
    };
    cx<SC> rho0 = {SC(1), SC(0)}, alpha = {SC(0), SC(0)}, omega = {SC(1), SC(0)};
    double bn2 = -1;
    int cycle = 0;
    for (;; ++cycle) {
        // |R0|^2 and rho1 = <rt, R0> in one reduction
        {
            cx<TC> v[2] = {czero<TC>(), czero<TC>()};
            for (int i = r0 + tid; i < r1; i += kThreads) {
                cx<TC> ri = ld<TC>(a.R[0], i);
                v[0].re += norm2(ri);
                v[1] = v[1] + cmulc(ld<TC>(a.rt, i), ri);
            }
            if (!grid_reduce<2, TC>(a, v, 2, red_sh, res)) return;
        }
        const double rn2 = res[0].re;
        if (bn2 < 0) bn2 = rn2;
        if (!(rn2 == rn2)) {   // NaN
            if (blockIdx.x == 0 && tid == 0) atomicExch(&a.bar->err, 2);
            return;
        }
        if (rn2 <= a.tol * a.tol * bn2 || cycle >= a.maxit) break;
        cx<SC> rho1 = ccast<SC>(res[1]);
        rho0 = SC(-1) * omega * rho0;
        for (int j = 0; j < ell; ++j) {
            const cx<SC> beta = cdiv(alpha * rho1, rho0);
            rho0 = rho1;
            for (int i = r0 + tid; i < r1; i += kThreads)
                for (int q = 0; q <= j; ++q) {
                    cx<TC> u = ld<TC>(a.U[q], i);
                    st<TC>(a.U[q], i, ld<TC>(a.R[q], i) - ccast<TC>(beta) * u);
                }
            if (!grid_sync(a.bar)) return;
            // U_{j+1} = A U_j and gamma = <rt, U_{j+1}>
            {
                cx<TC> v[1] = {czero<TC>()};
                if (!stencil_rows<TC, BF>(a, rg, xbuf, a.U[j], a.U[j + 1], a.rt, r0, r1, v[0])) {
                    atomicExch(&a.bar->err, 1);
                    return;
                }
                if (!grid_reduce<1, TC>(a, v, 1, red_sh, res)) return;
            }
            alpha = cdiv(rho0, ccast<SC>(res[0]));
            for (int i = r0 + tid; i < r1; i += kThreads) {
                for (int q = 0; q <= j; ++q)
                    st<TC>(a.R[q], i, ld<TC>(a.R[q], i) - ccast<TC>(alpha) * ld<TC>(a.U[q + 1], i));
                st<TC>(a.x, i, ld<TC>(a.x, i) + ccast<TC>(alpha) * ld<TC>(a.U[0], i));
            }
            if (!grid_sync(a.bar)) return;
            // R_{j+1} = A R_j; the next BiCG step needs rho1 = <rt, R_{j+1}>
            {
                cx<TC> v[1] = {czero<TC>()};
                if (!stencil_rows<TC, BF>(a, rg, xbuf, a.R[j], a.R[j + 1], a.rt, r0, r1, v[0])) {
                    atomicExch(&a.bar->err, 1);
                    return;
                }
                if (j + 1 < ell) {
                    if (!grid_reduce<1, TC>(a, v, 1, red_sh, res)) return;
                    rho1 = ccast<SC>(res[0]);
                }
            }
        }
        // minimal-residual part from the Gram matrix G_pq = <R_p, R_q>, p, q = 0..ell
        {
            cx<TC> v[kMaxQ];
            int nq = (ell + 1) * (ell + 1);
            for (int q = 0; q < nq; ++q) v[q] = czero<TC>();
            for (int i = r0 + tid; i < r1; i += kThreads) {
                cx<TC> rv[kMaxEll + 1];
                for (int p = 0; p <= ell; ++p) rv[p] = ld<TC>(a.R[p], i);
                for (int p = 0; p <= ell; ++p)
                    for (int q = p; q <= ell; ++q) v[p * (ell + 1) + q] = v[p * (ell + 1) + q] + cmulc(rv[p], rv[q]);
            }
            if (!grid_reduce<kMaxQ, TC>(a, v, nq, red_sh, res)) return;
        }
        // Gram-Schmidt of R_1..R_ell expressed in the original basis:
        // Rt_j = sum_k C[j][k] R_k (k = 1..j), tau_ij = <Rt_i, Rt_j>/sigma_i.
        // One thread evaluates the scalar algebra; the update coefficients are
        // broadcast through shared memory.
        __shared__ cx<double> s_cx[kMaxEll + 1], s_cr[kMaxEll + 1], s_g[kMaxEll + 1];
        __shared__ int s_bad;
        // scalars in the solver's precision (FP32 for the FP32 coarse solve)
        using ST = TC;
        if (tid == 0) {
            cx<ST> C[kMaxEll + 1][kMaxEll + 1];
            ST sigma[kMaxEll + 1];
            cx<ST> gp[kMaxEll + 1], g[kMaxEll + 1], gpp[kMaxEll + 1], tau[kMaxEll + 1][kMaxEll + 1];
            auto G = [&](int p, int q) -> cx<ST> {   // <R_p, R_q>
                return ccast<ST>(p <= q ? res[p * (ell + 1) + q] : conj(res[q * (ell + 1) + p]));
            };
            // loops run to the compile-time bound kMaxEll with guards, in the same order as
            // the algorithm's loops to ell, so that every array lives in registers
#pragma unroll
            for (int j = 0; j <= kMaxEll; ++j)
#pragma unroll
                for (int k = 0; k <= kMaxEll; ++k) C[j][k] = czero<ST>();
            int bad = 0;
#pragma unroll
            for (int j = 1; j <= kMaxEll; ++j) {
                if (j > ell) break;
                C[j][j] = {1, 0};
#pragma unroll
                for (int i = 1; i < j; ++i) {
                    cx<ST> t = czero<ST>();
#pragma unroll
                    for (int p = 1; p <= i; ++p)
#pragma unroll
                        for (int q = 1; q <= j; ++q) t = t + conj(C[i][p]) * C[j][q] * G(p, q);
                    tau[i][j] = (ST(1) / sigma[i]) * t;
#pragma unroll
                    for (int k = 1; k <= i; ++k) C[j][k] = C[j][k] - tau[i][j] * C[i][k];
                }
                ST sg = 0;
                cx<ST> t0 = czero<ST>();
#pragma unroll
                for (int p = 1; p <= j; ++p) {
#pragma unroll
                    for (int q = 1; q <= j; ++q) sg += (conj(C[j][p]) * C[j][q] * G(p, q)).re;
                    t0 = t0 + conj(C[j][p]) * G(p, 0);
                }
                sigma[j] = sg;
                if (!(sg > 0)) bad = 1;
                gp[j] = (ST(1) / (sg > 0 ? sg : ST(1))) * t0;
            }
#pragma unroll
            for (int j = 0; j <= kMaxEll; ++j) g[j] = gpp[j] = czero<ST>();
#pragma unroll
            for (int j = 1; j <= kMaxEll; ++j)
                if (j == ell) g[j] = gp[j];
#pragma unroll
            for (int j = kMaxEll - 1; j >= 1; --j) {
                if (j >= ell) continue;
                cx<ST> t = gp[j];
#pragma unroll
                for (int i = j + 1; i <= kMaxEll; ++i)
                    if (i <= ell) t = t - tau[j][i] * g[i];
                g[j] = t;
            }
#pragma unroll
            for (int j = 1; j < kMaxEll; ++j) {
                if (j >= ell) break;
                cx<ST> t = g[j + 1];
#pragma unroll
                for (int i = j + 1; i < kMaxEll; ++i)
                    if (i < ell) t = t + tau[j][i] * g[i + 1];
                gpp[j] = t;
            }
            // x += g1 R0 + sum_{j<ell} gpp_j Rt_j ; R0 -= sum_j gp_j Rt_j ; U0 -= sum_j g_j U_j
            cx<ST> tx[kMaxEll + 1], tr[kMaxEll + 1];
#pragma unroll
            for (int k = 0; k <= kMaxEll; ++k) tx[k] = tr[k] = czero<ST>();
            tx[0] = g[1];
#pragma unroll
            for (int j = 1; j < kMaxEll; ++j)
#pragma unroll
                for (int k = 1; k <= j; ++k)
                    if (j < ell) tx[k] = tx[k] + gpp[j] * C[j][k];
#pragma unroll
            for (int j = 1; j <= kMaxEll; ++j)
#pragma unroll
                for (int k = 1; k <= j; ++k)
                    if (j <= ell) tr[k] = tr[k] + gp[j] * C[j][k];
#pragma unroll
            for (int k = 0; k <= kMaxEll; ++k) {
                if (k > ell) break;
                s_cx[k] = ccast<double>(tx[k]);
                s_cr[k] = ccast<double>(tr[k]);
                s_g[k] = ccast<double>(g[k]);
            }
            s_bad = bad;
        }
        __syncthreads();
        if (s_bad) {
            if (blockIdx.x == 0 && tid == 0) atomicExch(&a.bar->err, 2);
            return;
        }
        omega = ccast<SC>(s_g[ell]);
        cx<SC> cx_[kMaxEll + 1], cr[kMaxEll + 1], g[kMaxEll + 1];
#pragma unroll
        for (int k = 0; k <= kMaxEll; ++k) {
            cx_[k] = k <= ell ? ccast<SC>(s_cx[k]) : czero<SC>();
            cr[k] = k <= ell ? ccast<SC>(s_cr[k]) : czero<SC>();
            g[k] = k <= ell ? ccast<SC>(s_g[k]) : czero<SC>();
        }
        for (int i = r0 + tid; i < r1; i += kThreads) {
            cx<TC> xv = ld<TC>(a.x, i), r0v = ld<TC>(a.R[0], i), u0 = ld<TC>(a.U[0], i);
            xv = xv + ccast<TC>(cx_[0]) * r0v;
#pragma unroll
            for (int k = 1; k <= kMaxEll; ++k) {
                if (k > ell) break;
                cx<TC> rk = ld<TC>(a.R[k], i);
                xv = xv + ccast<TC>(cx_[k]) * rk;
                r0v = r0v - ccast<TC>(cr[k]) * rk;
                u0 = u0 - ccast<TC>(g[k]) * ld<TC>(a.U[k], i);
            }
            st<TC>(a.x, i, xv);
            st<TC>(a.R[0], i, r0v);
            st<TC>(a.U[0], i, u0);
        }
    }
    if (blockIdx.x == 0 && tid == 0) a.bar->cycles += cycle;
}

// one CTA per SM (152 barrier participants on GB300), if the kernel fits
int coop_grid(const void* fn, int smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kThreads, smem);
    if (per < 1) return 0;
    return sms;
}

}  // namespace

size_t coarse_solver_state_bytes() { return sizeof(GridBar) + 64; }
size_t coarse_solver_partial_bytes() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sizeof(double2) * (size_t)kMaxQ * sms;
}

cudaError_t launch_coarse_bicgstab(int cprec, const GeomH& gc, int nc, const void* B, const void* b, void* x,
                                   void* rt, void* const* R, void* const* U, int ell, double tol, int maxit,
                                   void* part, void* state, int cluster, cudaStream_t s) {
    if (ell < 1 || ell > kMaxEll) return cudaErrorInvalidValue;
    Args a;
    for (int i = 0; i < 4; ++i) a.L[i] = gc.L[i];
    a.Vc = gc.V;
    a.nc = nc;
    a.ell = ell;
    a.maxit = maxit;
    a.tol = tol;
    a.B = B;
    a.b = b;
    a.x = x;
    a.rt = rt;
    for (int j = 0; j <= kMaxEll; ++j) {
        a.R[j] = j <= ell ? R[j] : nullptr;
        a.U[j] = j <= ell ? U[j] : nullptr;
    }
    a.part = (double2*)part;
    a.bar = (GridBar*)state;
    if (nc % 2 != 0) return cudaErrorInvalidValue;
    // cprec: 0 FP64, 1 FP32, 2 FP32 vectors with a bfloat16 operator
    const int eb = cprec == 0 ? 16 : 8;
    a.row_bytes = 9 * nc * (cprec == 2 ? 4 : eb);
    if (a.row_bytes % 16 != 0) return cudaErrorInvalidValue;   // bulk copies move 16-byte multiples
    a.rows_per_chunk = kChunkBytes / a.row_bytes;
    if (a.rows_per_chunk < 1) return cudaErrorInvalidValue;   // nc too large for a ring slot
    if (a.rows_per_chunk > kMaxRowsPerWarp * kWarps) a.rows_per_chunk = kMaxRowsPerWarp * kWarps;
    a.sites_per_chunk = (a.rows_per_chunk - 1) / nc + 2;
    a.xseg_bytes = nc * eb;
    a.slot_bytes = kChunkBytes;
    const void* fn = cprec == 0   ? (const void*)coarse_bicgstab_kernel<double, false>
                     : cprec == 1 ? (const void*)coarse_bicgstab_kernel<float, false>
                                  : (const void*)coarse_bicgstab_kernel<float, true>;
    const int smem = kStages * (kChunkBytes + 9 * a.sites_per_chunk * a.xseg_bytes);
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void* params[] = {&a};
    if (cluster > 0) {
        // one thread-block cluster: its CTAs are co-scheduled by the hardware,
        // so the kernel's grid barrier is safe next to other kernels (several
        // such solves may run at once on different streams or graph branches)
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int cl = cluster > 8 ? 8 : cluster;
        for (; cl > 1; cl /= 2) {   // largest power-of-two cluster that fits
            at[0].val.clusterDim.x = cl;
            cfg.gridDim = dim3(cl);
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) == cudaSuccess && nclusters > 0) break;
            cudaGetLastError();
        }
        at[0].val.clusterDim.x = cl;
        cfg.gridDim = dim3(cl);
        note_launch();
        return cudaLaunchKernelExC(&cfg, fn, params);
    }
    int grid = coop_grid(fn, smem);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    note_launch();
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), params, smem, s);
}
