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
// straight from global memory into registers (coalesced 16-byte words, two
// rows per warp in flight), so the operator never passes through shared
// memory; the neighbour blocks of the CTA's coarse sites are gathered into
// shared memory once per pass.
//
// Grid barriers spin with a bounded count; on timeout the
// kernel records AMG_TIMEOUT in the status word and every CTA returns.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxEll = 4;
constexpr int kMaxQ = (kMaxEll + 1) * (kMaxEll + 1) + 2;   // reduced quantities per barrier
constexpr long long kSpinLimit = 40000000;                    // ~ seconds of polling
constexpr int kU = 7;                                         // 16-byte operator words per lane in flight per row
constexpr int kXBytes = 96 * 1024;                            // shared memory for one group's neighbour blocks

struct GridBar {
    unsigned count;   // barrier word: arrivals in the low bits, a phase bit on top
    unsigned pad;
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
    int row_bytes;   // 9 * nc * (bytes per operator entry), a multiple of 16
    int xgroup;      // coarse sites whose neighbour blocks are staged in shared memory at once
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

// grid barrier on one word: CTA 0 adds 2^31 - (nCTA - 1), every other CTA
// adds 1, so the top bit flips exactly when the last CTA arrives and the low
// bits return to their value (the scheme of cooperative groups' grid sync).
// One acquire-release atomic per CTA, then a bounded spin on the top bit; the
// CTA's writes are published by __syncthreads + the releasing atomic.
// Returns false if it gave up (then the caller returns).
DEV bool grid_sync(GridBar* gb) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int* verr = &gb->err;
        const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
        const unsigned old = atom_add_acqrel(&gb->count, inc);
        int ok = 1;
        long long it = 0;
        while (((ld_acquire(&gb->count) ^ old) & 0x80000000u) == 0) {
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

// one 16-byte word of an operator row: 2 FP32 complex entries, 4 bfloat16
// complex entries (BF16 storage, FP32 arithmetic) or 1 FP64 complex entry,
// multiplied into acc with the matching entries x[0 .. per-1] of the row's
// neighbour block (shared memory, 16-byte aligned)
template <typename TC, int ST> struct OpWord;   // ST: 0 as TC, 1 bfloat16, 2 FP32 widened to FP64
template <> struct OpWord<float, 0> {
    static constexpr int per = 2;
    DEV static void mac(uint4 v, const cx<float>* x, cx<float>& acc) {
        const float4 o = make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z),
                                     __uint_as_float(v.w));
        const float4 xv = *reinterpret_cast<const float4*>(x);
        cfma(acc, cx<float>{o.x, o.y}, cx<float>{xv.x, xv.y});
        cfma(acc, cx<float>{o.z, o.w}, cx<float>{xv.z, xv.w});
    }
};
template <> struct OpWord<float, 1> {
    static constexpr int per = 4;
    DEV static void mac(uint4 v, const cx<float>* x, cx<float>& acc) {
        const unsigned u[4] = {v.x, v.y, v.z, v.w};
        const float4 x01 = *reinterpret_cast<const float4*>(x), x23 = *reinterpret_cast<const float4*>(x + 2);
        const float xs[8] = {x01.x, x01.y, x01.z, x01.w, x23.x, x23.y, x23.z, x23.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 o = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u[e]));
            cfma(acc, cx<float>{o.x, o.y}, cx<float>{xs[2 * e], xs[2 * e + 1]});
        }
    }
};
template <> struct OpWord<double, 2> {   // FP32-exact entries stored in FP32, FP64 arithmetic
    static constexpr int per = 2;
    DEV static void mac(uint4 v, const cx<double>* x, cx<double>& acc) {
        const double2 x0 = *reinterpret_cast<const double2*>(x), x1 = *reinterpret_cast<const double2*>(x + 1);
        cfma(acc, cx<double>{(double)__uint_as_float(v.x), (double)__uint_as_float(v.y)}, cx<double>{x0.x, x0.y});
        cfma(acc, cx<double>{(double)__uint_as_float(v.z), (double)__uint_as_float(v.w)}, cx<double>{x1.x, x1.y});
    }
};
template <> struct OpWord<double, 0> {
    static constexpr int per = 1;
    DEV static void mac(uint4 v, const cx<double>* x, cx<double>& acc) {
        const double2 o = make_double2(__hiloint2double((int)v.y, (int)v.x), __hiloint2double((int)v.w, (int)v.z));
        const double2 xv = *reinterpret_cast<const double2*>(x);
        cfma(acc, cx<double>{o.x, o.y}, cx<double>{xv.x, xv.y});
    }
};

// y(row) = sum_{d,col} B[row][d][col] x(nbr(X, d))[col] for the rows [r0, r1)
// of this CTA; returns the per-thread partial <w, y> in dotp (w != nullptr).
// The CTA's sites are taken in groups of a.xgroup: the nine neighbour blocks
// of every site of the group are gathered into shared memory (generic loads
// through L2, since other CTAs wrote the vector), then each warp computes two
// rows at a time, streaming their operator words straight from global memory
// into registers (kU coalesced 16-byte loads per lane and row in flight) --
// the operator is read exactly once and never passes through shared memory.
// Contains __syncthreads(): called by all threads of the CTA.
template <typename TC, int BF>
DEV void stencil_rows(const Args& a, cx<TC>* xbuf, int* nbr, const void* xin, void* yout, const void* w, int r0,
                      int r1, cx<TC>& dotp) {
    using W = OpWord<TC, BF>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    const int nc = a.nc, K = 9 * nc, nw = K / W::per;
    const int wseg = nc * (int)sizeof(cx<TC>) / 16;   // 16-byte words per neighbour segment
    const int Xa = r0 / nc, Xb = r1 > r0 ? (r1 - 1) / nc : Xa - 1;
    for (int Xg = Xa; Xg <= Xb; Xg += a.xgroup) {
        const int gs = min(a.xgroup, Xb - Xg + 1);
        __syncthreads();   // the previous group's blocks are no longer read
        for (int t = tid; t < gs * 9; t += kThreads) nbr[t] = coarse_neighbour(a, Xg + t / 9, t % 9);
        __syncthreads();
        {
            const uint4* xg = (const uint4*)xin;
            uint4* xs = (uint4*)xbuf;
            for (int p = tid; p < gs * 9 * wseg; p += kThreads) {
                const int sd = p / wseg, q = p - sd * wseg;
                xs[p] = __ldcg(xg + (size_t)nbr[sd] * wseg + q);
            }
        }
        __syncthreads();
        const int ra = max(r0, Xg * nc), rb = min(r1, (Xg + gs) * nc);
        for (int rA = ra + 2 * warp; rA < rb; rA += 2 * kWarps) {
            const int rB = rA + 1;
            const bool hasB = rB < rb;
            cx<TC> wA = czero<TC>(), wB = czero<TC>();
            if (w && lane == 0) {   // loaded now, used after the row sums
                wA = ld<TC>(w, rA);
                if (hasB) wB = ld<TC>(w, rB);
            }
            const uint4* opA = (const uint4*)((const unsigned char*)a.B + (size_t)rA * a.row_bytes);
            const uint4* opB = opA + nw;
            const cx<TC>* xA = xbuf + (size_t)(rA / nc - Xg) * K;
            const cx<TC>* xB = xbuf + (size_t)(rB / nc - Xg) * K;
            cx<TC> accA = czero<TC>(), accB = czero<TC>();
            for (int k0 = 0; k0 < nw; k0 += 32 * kU) {
                uint4 va[kU], vb[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int k = k0 + lane + 32 * u;
                    va[u] = k < nw ? __ldg(opA + k) : make_uint4(0u, 0u, 0u, 0u);
                    vb[u] = (hasB && k < nw) ? __ldg(opB + k) : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int k = k0 + lane + 32 * u;
                    if (k < nw) {
                        W::mac(va[u], xA + (size_t)k * W::per, accA);
                        if (hasB) W::mac(vb[u], xB + (size_t)k * W::per, accB);
                    }
                }
            }
            accA.re = warp_sum(accA.re);
            accA.im = warp_sum(accA.im);
            accB.re = warp_sum(accB.re);
            accB.im = warp_sum(accB.im);
            if (lane == 0) {
                st<TC>(yout, rA, accA);
                if (hasB) st<TC>(yout, rB, accB);
                if (w) dotp = dotp + cmulc(wA, accA) + cmulc(wB, accB);
            }
        }
    }
}

template <typename TC, int BF>
__global__ void __launch_bounds__(kThreads) coarse_bicgstab_kernel(Args a) {
    __shared__ cx<double> red_sh[kMaxQ * kWarps];
    __shared__ cx<double> res[kMaxQ];
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    cx<TC>* xbuf = (cx<TC>*)dyn_smem;                                    // xgroup x 9 neighbour blocks
    int* nbr = (int*)(dyn_smem + (size_t)a.xgroup * 9 * a.nc * sizeof(cx<TC>));   // their sites
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
                stencil_rows<TC, BF>(a, xbuf, nbr, a.U[j], a.U[j + 1], a.rt, r0, r1, v[0]);
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
                stencil_rows<TC, BF>(a, xbuf, nbr, a.R[j], a.R[j + 1], a.rt, r0, r1, v[0]);
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
    // cprec: 0 FP64, 1 FP32, 2 FP32 vectors with a bfloat16 operator, 3 FP64 vectors with an
    // FP32-stored operator (FP32-exact entries)
    if (cprec < 0 || cprec > 3) return cudaErrorInvalidValue;
    const int eb = (cprec == 0 || cprec == 3) ? 16 : 8;                        // vector entry
    a.row_bytes = 9 * nc * (cprec == 2 ? 4 : cprec == 3 ? 8 : eb);             // operator entry
    if (a.row_bytes % 16 != 0) return cudaErrorInvalidValue;   // rows are read in 16-byte words
    const int block_bytes = 9 * nc * eb;                                  // one site's neighbour blocks
    a.xgroup = kXBytes / block_bytes;
    if (a.xgroup < 1) return cudaErrorInvalidValue;
    const void* fn = cprec == 0   ? (const void*)coarse_bicgstab_kernel<double, 0>
                     : cprec == 3 ? (const void*)coarse_bicgstab_kernel<double, 2>
                     : cprec == 1 ? (const void*)coarse_bicgstab_kernel<float, 0>
                                  : (const void*)coarse_bicgstab_kernel<float, 1>;
    const int smem = a.xgroup * (block_bytes + 9 * (int)sizeof(int));
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
