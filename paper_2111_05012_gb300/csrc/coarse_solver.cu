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
// Several right-hand sides (up to kMaxNB) are solved in lockstep by one
// launch: every stencil pass streams each operator word once and applies it
// to all of them, while the BiCGStab(l) scalars, the stopping test and the
// vector updates stay per right-hand side, so each one follows exactly the
// iterates of its own single solve (same rows per CTA, same summation order).
// A right-hand side that has converged is frozen (no more updates of its
// vectors or scalars) while the others go on.
//
// Grid barriers spin with a bounded count; on timeout the
// kernel records AMG_TIMEOUT in the status word and every CTA returns.
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxEll = 4;
constexpr int kMaxNB = 4;                                   // right-hand sides per launch
constexpr int kMaxQ = (kMaxEll + 1) * (kMaxEll + 1) + 2;   // reduced quantities per barrier (>= 2 kMaxNB)
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
    int nb;          // right-hand sides of this launch; vector r of a field starts r * Vc * nc entries in
    double tol;
    const void* B;
    const void* b;
    void* x;
    void* rt;
    void* R[kMaxEll + 1];
    void* U[kMaxEll + 1];
    double2* part;   // [kMaxQ][ncta]
    GridBar* bar;
    int row_bytes;   // 9 * nc * (bytes per operator entry), a multiple of 16
    int xgroup;      // coarse sites whose neighbour blocks are staged in shared memory at once
    int cta, ncta;   // this CTA's index among the solve's CTAs and their number (the grid, or one
                     // cluster of a launch that solves several problems, one per cluster)
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
DEV bool grid_sync(GridBar* gb, int cta, int ncta) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int* verr = &gb->err;
        const unsigned inc = cta == 0 ? 0x80000000u - ((unsigned)ncta - 1u) : 1u;
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
        a.part[(size_t)threadIdx.x * a.ncta + a.cta] = make_double2(t.re, t.im);
    }
    if (!grid_sync(a.bar, a.cta, a.ncta)) return false;
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
            t[k] = i < a.ncta ? __ldcg(a.part + (size_t)q * a.ncta + i) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            re += t[k].x;
            im += t[k].y;
        }
        for (int i = lane + 32 * kPer; i < a.ncta; i += 32) {
            double2 u = __ldcg(a.part + (size_t)q * a.ncta + i);
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
DEV void my_rows(int nrows, int cta, int ncta, int& r0, int& r1) {
    int per = (nrows + ncta - 1) / ncta;
    r0 = cta * per;
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

// y_r(row) = sum_{d,col} B[row][d][col] x_r(nbr(X, d))[col] for the rows [r0, r1)
// of this CTA and the a.nb right-hand sides r; returns the per-thread partials
// <w_r, y_r> in dotp[r] (w != nullptr).  The CTA's sites are taken in groups of
// a.xgroup: the nine neighbour blocks of every site of the group are gathered
// into shared memory for every right-hand side (generic loads through L2,
// since other CTAs wrote the vectors), then each warp computes two rows at a
// time, streaming their operator words straight from global memory into
// registers (kU coalesced 16-byte loads per lane and row in flight) and
// applying each word to all right-hand sides -- the operator is read exactly
// once per pass and never passes through shared memory.
// Contains __syncthreads(): called by all threads of the CTA.
template <typename TC, int BF, int NB>
DEV void stencil_rows(const Args& a, cx<TC>* xbuf, int* nbr, const void* xin, void* yout, const void* w, int r0,
                      int r1, cx<TC> (&dotp)[NB]) {
    using W = OpWord<TC, BF>;
    // operator words in flight per lane and row: each word feeds NB right-hand sides, so fewer
    // are needed to cover the latency (and the accumulators take the registers)
    constexpr int KU = NB == 1 ? kU : NB == 2 ? 4 : 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    const int nc = a.nc, K = 9 * nc, nw = K / W::per, nb = a.nb;
    const size_t n = (size_t)a.Vc * nc;                     // entries per vector
    const int wseg = nc * (int)sizeof(cx<TC>) / 16;   // 16-byte words per neighbour segment
    const size_t wvec = n * sizeof(cx<TC>) / 16;       // 16-byte words per vector
    const int xs_r = a.xgroup * K;                     // xbuf entries per right-hand side
    const int Xa = r0 / nc, Xb = r1 > r0 ? (r1 - 1) / nc : Xa - 1;
    for (int Xg = Xa; Xg <= Xb; Xg += a.xgroup) {
        const int gs = min(a.xgroup, Xb - Xg + 1);
        __syncthreads();   // the previous group's blocks are no longer read
        for (int t = tid; t < gs * 9; t += kThreads) nbr[t] = coarse_neighbour(a, Xg + t / 9, t % 9);
        __syncthreads();
        {
            const uint4* xg = (const uint4*)xin;
            uint4* xs = (uint4*)xbuf;
            const int per_r = gs * 9 * wseg;
            for (int p = tid; p < nb * per_r; p += kThreads) {
                const int r = p / per_r, pp = p - r * per_r;
                const int sd = pp / wseg, q = pp - sd * wseg;
                xs[(size_t)r * (xs_r * sizeof(cx<TC>) / 16) + pp] = __ldcg(xg + r * wvec + (size_t)nbr[sd] * wseg + q);
            }
        }
        __syncthreads();
        const int ra = max(r0, Xg * nc), rb = min(r1, (Xg + gs) * nc);
        for (int rA = ra + 2 * warp; rA < rb; rA += 2 * kWarps) {
            const int rB = rA + 1;
            const bool hasB = rB < rb;
            cx<TC> wA1 = czero<TC>(), wB1 = czero<TC>();
            if (NB == 1 && w && lane == 0) {   // loaded now, used after the row sums
                wA1 = ld<TC>(w, rA);
                if (hasB) wB1 = ld<TC>(w, rB);
            }
            const uint4* opA = (const uint4*)((const unsigned char*)a.B + (size_t)rA * a.row_bytes);
            const uint4* opB = opA + nw;
            const cx<TC>* xA = xbuf + (size_t)(rA / nc - Xg) * K;
            const cx<TC>* xB = xbuf + (size_t)(rB / nc - Xg) * K;
            cx<TC> accA[NB], accB[NB];
#pragma unroll
            for (int r = 0; r < NB; ++r) accA[r] = accB[r] = czero<TC>();
            for (int k0 = 0; k0 < nw; k0 += 32 * KU) {
                uint4 va[KU], vb[KU];
#pragma unroll
                for (int u = 0; u < KU; ++u) {
                    const int k = k0 + lane + 32 * u;
                    va[u] = k < nw ? __ldg(opA + k) : make_uint4(0u, 0u, 0u, 0u);
                    vb[u] = (hasB && k < nw) ? __ldg(opB + k) : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (int u = 0; u < KU; ++u) {
                    const int k = k0 + lane + 32 * u;
                    if (k < nw) {
#pragma unroll
                        for (int r = 0; r < NB; ++r) {
                            if (r < nb) {
                                W::mac(va[u], xA + (size_t)r * xs_r + (size_t)k * W::per, accA[r]);
                                if (hasB) W::mac(vb[u], xB + (size_t)r * xs_r + (size_t)k * W::per, accB[r]);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                if (r >= nb) break;
                accA[r].re = warp_sum(accA[r].re);
                accA[r].im = warp_sum(accA[r].im);
                accB[r].re = warp_sum(accB[r].re);
                accB[r].im = warp_sum(accB[r].im);
                if (lane == 0) {
                    st<TC>(yout, r * n + rA, accA[r]);
                    if (hasB) st<TC>(yout, r * n + rB, accB[r]);
                    if (w) {
                        const cx<TC> wa = NB == 1 ? wA1 : ld<TC>(w, r * n + rA);
                        const cx<TC> wb = NB == 1 ? wB1 : (hasB ? ld<TC>(w, r * n + rB) : czero<TC>());
                        dotp[r] = dotp[r] + cmulc(wa, accA[r]) + cmulc(wb, accB[r]);
                    }
                }
            }
        }
    }
}

// Scalar algebra of the minimal-residual part for one right-hand side from its
// Gram matrix G_pq = <R_p, R_q> (res, packed upper triangle p <= q): Gram-Schmidt
// of R_1..R_ell expressed in the original basis, Rt_j = sum_k C[j][k] R_k
// (k = 1..j), tau_ij = <Rt_i, Rt_j>/sigma_i; writes the update coefficients of
// x, R_0 and U_0.  Runs in one thread, in the solver's precision ST.  Returns
// false on a breakdown (sigma_j <= 0).
template <typename ST>
DEV bool mr_coefficients(const cx<double>* res, int ell, cx<double>* out_x, cx<double>* out_r, cx<double>* out_g) {
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
    bool ok = true;
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
        if (!(sg > 0)) ok = false;
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
        out_x[k] = ccast<double>(tx[k]);
        out_r[k] = ccast<double>(tr[k]);
        out_g[k] = ccast<double>(g[k]);
    }
    return ok;
}

template <typename TC, int BF, int NB>
DEV void coarse_bicgstab_body(Args& a) {
    using SC = TC;   // BiCG scalars in the solver's precision
    __shared__ cx<double> red_sh[kMaxQ * kWarps];
    __shared__ cx<double> res[kMaxQ];
    // per right-hand side scalars, owned by thread 0 (kept as doubles: exact for SC = float too)
    __shared__ cx<double> s_rho0[NB], s_rho1[NB], s_alpha[NB], s_omega[NB], s_beta[NB];
    __shared__ double s_bn2[NB];
    __shared__ int s_act[NB], s_any, s_bad;
    __shared__ cx<double> s_cx[NB][kMaxEll + 1], s_cr[NB][kMaxEll + 1], s_g[NB][kMaxEll + 1];
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    cx<TC>* xbuf = (cx<TC>*)dyn_smem;   // [NB][xgroup x 9 neighbour blocks]
    int* nbr = (int*)(dyn_smem + (size_t)NB * a.xgroup * 9 * a.nc * sizeof(cx<TC>));   // their sites
    const int ell = a.ell, nb = a.nb;
    const size_t n = (size_t)a.Vc * a.nc;
    int r0, r1;
    my_rows((int)n, a.cta, a.ncta, r0, r1);
    const int tid = threadIdx.x;
    // initial state: x = 0, R0 = b, rt = b, U0 = 0
    for (int r = 0; r < nb; ++r)
        for (int i = r0 + tid; i < r1; i += kThreads) {
            const size_t k = r * n + i;
            cx<TC> bi = ld<TC>(a.b, k);
            st<TC>(a.x, k, czero<TC>());
            st<TC>(a.R[0], k, bi);
            st<TC>(a.rt, k, bi);
            st<TC>(a.U[0], k, czero<TC>());
        }
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
    if (tid < NB) {
        s_rho0[tid] = s_rho1[tid] = s_omega[tid] = {1.0, 0.0};
        s_alpha[tid] = s_beta[tid] = {0.0, 0.0};
        s_bn2[tid] = -1;
        s_act[tid] = tid < nb;
    }
    __syncthreads();
    int cycle = 0;
    for (;; ++cycle) {
        // |R0|^2 and rho1 = <rt, R0> of every right-hand side in one reduction
        {
            cx<TC> v[2 * NB];
#pragma unroll
            for (int q = 0; q < 2 * NB; ++q) v[q] = czero<TC>();
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                if (r >= nb) break;
                for (int i = r0 + tid; i < r1; i += kThreads) {
                    cx<TC> ri = ld<TC>(a.R[0], r * n + i);
                    v[2 * r].re += norm2(ri);
                    v[2 * r + 1] = v[2 * r + 1] + cmulc(ld<TC>(a.rt, r * n + i), ri);
                }
            }
            if (!grid_reduce<2 * NB, TC>(a, v, 2 * nb, red_sh, res)) return;
        }
        if (tid == 0) {
            int any = 0, bad = 0;
            for (int r = 0; r < nb; ++r) {
                if (!s_act[r]) continue;
                const double rn2 = res[2 * r].re;
                if (s_bn2[r] < 0) s_bn2[r] = rn2;
                if (!(rn2 == rn2)) bad = 1;   // NaN
                if (rn2 <= a.tol * a.tol * s_bn2[r] || cycle >= a.maxit) {
                    s_act[r] = 0;   // converged (or out of cycles): frozen from here on
                    continue;
                }
                any = 1;
                s_rho1[r] = ccast<double>(ccast<SC>(res[2 * r + 1]));
                s_rho0[r] = ccast<double>(SC(-1) * ccast<SC>(s_omega[r]) * ccast<SC>(s_rho0[r]));
            }
            s_any = any;
            s_bad = bad;
        }
        __syncthreads();
        if (s_bad) {
            if (a.cta == 0 && tid == 0) atomicExch(&a.bar->err, 2);
            return;
        }
        if (!s_any) break;
        for (int j = 0; j < ell; ++j) {
            if (tid == 0)
                for (int r = 0; r < nb; ++r) {
                    if (!s_act[r]) continue;
                    s_beta[r] = ccast<double>(
                        cdiv(ccast<SC>(s_alpha[r]) * ccast<SC>(s_rho1[r]), ccast<SC>(s_rho0[r])));
                    s_rho0[r] = s_rho1[r];
                }
            __syncthreads();
            for (int r = 0; r < nb; ++r) {
                if (!s_act[r]) continue;
                const cx<TC> beta = ccast<TC>(s_beta[r]);
                for (int i = r0 + tid; i < r1; i += kThreads)
                    for (int q = 0; q <= j; ++q) {
                        cx<TC> u = ld<TC>(a.U[q], r * n + i);
                        st<TC>(a.U[q], r * n + i, ld<TC>(a.R[q], r * n + i) - beta * u);
                    }
            }
            if (!grid_sync(a.bar, a.cta, a.ncta)) return;
            // U_{j+1} = A U_j and gamma = <rt, U_{j+1}>
            {
                cx<TC> d[NB];
#pragma unroll
                for (int r = 0; r < NB; ++r) d[r] = czero<TC>();
                stencil_rows<TC, BF, NB>(a, xbuf, nbr, a.U[j], a.U[j + 1], a.rt, r0, r1, d);
                if (!grid_reduce<NB, TC>(a, d, nb, red_sh, res)) return;
            }
            if (tid == 0)
                for (int r = 0; r < nb; ++r)
                    if (s_act[r]) s_alpha[r] = ccast<double>(cdiv(ccast<SC>(s_rho0[r]), ccast<SC>(res[r])));
            __syncthreads();
            for (int r = 0; r < nb; ++r) {
                if (!s_act[r]) continue;
                const cx<TC> alpha = ccast<TC>(s_alpha[r]);
                for (int i = r0 + tid; i < r1; i += kThreads) {
                    const size_t k = r * n + i;
                    for (int q = 0; q <= j; ++q)
                        st<TC>(a.R[q], k, ld<TC>(a.R[q], k) - alpha * ld<TC>(a.U[q + 1], k));
                    st<TC>(a.x, k, ld<TC>(a.x, k) + alpha * ld<TC>(a.U[0], k));
                }
            }
            if (!grid_sync(a.bar, a.cta, a.ncta)) return;
            // R_{j+1} = A R_j; the next BiCG step needs rho1 = <rt, R_{j+1}>
            {
                cx<TC> d[NB];
#pragma unroll
                for (int r = 0; r < NB; ++r) d[r] = czero<TC>();
                stencil_rows<TC, BF, NB>(a, xbuf, nbr, a.R[j], a.R[j + 1], a.rt, r0, r1, d);
                if (j + 1 < ell) {
                    if (!grid_reduce<NB, TC>(a, d, nb, red_sh, res)) return;
                    if (tid == 0)
                        for (int r = 0; r < nb; ++r)
                            if (s_act[r]) s_rho1[r] = ccast<double>(ccast<SC>(res[r]));
                }
            }
        }
        // minimal-residual part from the Gram matrix G_pq = <R_p, R_q>, p, q = 0..ell, of
        // each active right-hand side (one reduction each); thread 0 evaluates the scalar
        // algebra and broadcasts the update coefficients through shared memory
        for (int r = 0; r < nb; ++r) {
            if (!s_act[r]) continue;
            cx<TC> v[kMaxQ];
            const int nq = (ell + 1) * (ell + 1);
            for (int q = 0; q < nq; ++q) v[q] = czero<TC>();
            for (int i = r0 + tid; i < r1; i += kThreads) {
                cx<TC> rv[kMaxEll + 1];
                for (int p = 0; p <= ell; ++p) rv[p] = ld<TC>(a.R[p], r * n + i);
                for (int p = 0; p <= ell; ++p)
                    for (int q = p; q <= ell; ++q) v[p * (ell + 1) + q] = v[p * (ell + 1) + q] + cmulc(rv[p], rv[q]);
            }
            if (!grid_reduce<kMaxQ, TC>(a, v, nq, red_sh, res)) return;
            if (tid == 0) {
                s_bad = mr_coefficients<SC>(res, ell, s_cx[r], s_cr[r], s_g[r]) ? 0 : 1;
                s_omega[r] = s_g[r][ell];
            }
            __syncthreads();
            if (s_bad) {
                if (a.cta == 0 && tid == 0) atomicExch(&a.bar->err, 2);
                return;
            }
        }
        for (int r = 0; r < nb; ++r) {
            if (!s_act[r]) continue;
            for (int i = r0 + tid; i < r1; i += kThreads) {
                const size_t kk = r * n + i;
                cx<TC> xv = ld<TC>(a.x, kk), r0v = ld<TC>(a.R[0], kk), u0 = ld<TC>(a.U[0], kk);
                xv = xv + ccast<TC>(s_cx[r][0]) * r0v;
#pragma unroll
                for (int k = 1; k <= kMaxEll; ++k) {
                    if (k > ell) break;
                    cx<TC> rk = ld<TC>(a.R[k], kk);
                    xv = xv + ccast<TC>(s_cx[r][k]) * rk;
                    r0v = r0v - ccast<TC>(s_cr[r][k]) * rk;
                    u0 = u0 - ccast<TC>(s_g[r][k]) * ld<TC>(a.U[k], kk);
                }
                st<TC>(a.x, kk, xv);
                st<TC>(a.R[0], kk, r0v);
                st<TC>(a.U[0], kk, u0);
            }
        }
    }
    if (a.cta == 0 && tid == 0) a.bar->cycles += cycle;
}

template <typename TC, int BF, int NB>
__global__ void __launch_bounds__(kThreads) coarse_bicgstab_kernel(Args a) {
    a.cta = blockIdx.x;
    a.ncta = gridDim.x;
    coarse_bicgstab_body<TC, BF, NB>(a);
}

// several independent problems in one launch: cluster c (csize CTAs) solves problem c with
// the arguments descs[c]; its barriers and reductions involve only its own CTAs
template <typename TC, int BF>
__global__ void __launch_bounds__(kThreads) coarse_bicgstab_multi_kernel(const Args* __restrict__ descs, int csize) {
    Args a = descs[blockIdx.x / csize];
    a.cta = blockIdx.x % csize;
    a.ncta = csize;
    coarse_bicgstab_body<TC, BF, 1>(a);
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

template <int NB> const void* solver_fn(int cprec) {
    return cprec == 0   ? (const void*)coarse_bicgstab_kernel<double, 0, NB>
           : cprec == 3 ? (const void*)coarse_bicgstab_kernel<double, 2, NB>
           : cprec == 1 ? (const void*)coarse_bicgstab_kernel<float, 0, NB>
                        : (const void*)coarse_bicgstab_kernel<float, 1, NB>;
}

}  // namespace

int coarse_solver_max_rhs() { return kMaxNB; }
int coarse_solver_max_xgroup(int cprec, int nc, int nb) {
    const int NB = nb <= 1 ? 1 : nb == 2 ? 2 : 4;
    const int eb = (cprec == 0 || cprec == 3) ? 16 : 8;
    return kXBytes / (9 * nc * eb * NB);
}

size_t coarse_solver_state_bytes() { return sizeof(GridBar) + 64; }
size_t coarse_solver_partial_bytes() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sizeof(double2) * (size_t)kMaxQ * sms;
}


// the kernel arguments of one solve and its dynamic shared memory (cudaSuccess if valid)
static cudaError_t make_args(Args& a, int& smem, int cprec, const GeomH& gc, int nc, const void* B, const void* b,
                             void* x, void* rt, void* const* R, void* const* U, int ell, double tol, int maxit,
                             void* part, void* state, int nb, int xgroup) {
    if (ell < 1 || ell > kMaxEll) return cudaErrorInvalidValue;
    if (nb < 1 || nb > kMaxNB) return cudaErrorInvalidValue;
    const int NB = nb == 1 ? 1 : nb == 2 ? 2 : 4;   // compiled batch widths
    a.nb = nb;
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
    a.xgroup = kXBytes / (block_bytes * NB);
    if (xgroup > 0 && xgroup < a.xgroup) a.xgroup = xgroup;
    if (a.xgroup < 1) return cudaErrorInvalidValue;
    smem = a.xgroup * (NB * block_bytes + 9 * (int)sizeof(int));
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    a.cta = 0;
    a.ncta = 1;
    return cudaSuccess;
}

cudaError_t launch_coarse_bicgstab(int cprec, const GeomH& gc, int nc, const void* B, const void* b, void* x,
                                   void* rt, void* const* R, void* const* U, int ell, double tol, int maxit,
                                   void* part, void* state, int cluster, cudaStream_t s, int nb, int xgroup) {
    Args a;
    int smem = 0;
    cudaError_t e = make_args(a, smem, cprec, gc, nc, B, b, x, rt, R, U, ell, tol, maxit, part, state, nb, xgroup);
    if (e != cudaSuccess) return e;
    const int NB = nb == 1 ? 1 : nb == 2 ? 2 : 4;
    const void* fn = NB == 1 ? solver_fn<1>(cprec) : NB == 2 ? solver_fn<2>(cprec) : solver_fn<4>(cprec);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
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

size_t coarse_solver_desc_bytes() { return sizeof(Args); }

cudaError_t launch_coarse_bicgstab_multi(const CoarseSolveDesc* d, int n, void* host_args, void* dev_args,
                                         cudaStream_t s) {
    if (n < 1) return cudaSuccess;
    const int cprec = d[0].cprec;
    Args* args = (Args*)host_args;
    int smem = 0;
    for (int i = 0; i < n; ++i) {
        if (d[i].cprec != cprec) return cudaErrorInvalidValue;   // one kernel instance for the launch
        int sm = 0;
        cudaError_t e = make_args(args[i], sm, d[i].cprec, d[i].gc, d[i].nc, d[i].B, d[i].b, d[i].x, d[i].rt, d[i].R,
                                  d[i].U, d[i].ell, d[i].tol, d[i].maxit, d[i].part, d[i].state, 1, d[i].xgroup);
        if (e != cudaSuccess) return e;
        smem = sm > smem ? sm : smem;
    }
    cudaError_t e = cudaMemcpyAsync(dev_args, args, sizeof(Args) * n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    const void* fn = cprec == 0   ? (const void*)coarse_bicgstab_multi_kernel<double, 0>
                     : cprec == 3 ? (const void*)coarse_bicgstab_multi_kernel<double, 2>
                     : cprec == 1 ? (const void*)coarse_bicgstab_multi_kernel<float, 0>
                                  : (const void*)coarse_bicgstab_multi_kernel<float, 1>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
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
    int cl = 8;
    for (; cl > 1; cl /= 2) {   // largest power-of-two cluster that fits
        at[0].val.clusterDim.x = cl;
        cfg.gridDim = dim3(cl);
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) == cudaSuccess && nclusters > 0) break;
        cudaGetLastError();
    }
    at[0].val.clusterDim.x = cl;
    cfg.gridDim = dim3(cl * n);
    const Args* dp = (const Args*)dev_args;
    int csize = cl;
    void* params[] = {&dp, &csize};
    note_launch();
    return cudaLaunchKernelExC(&cfg, fn, params);
}
