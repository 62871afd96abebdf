// C ABI of the library (include/lqcd_amg.h): handles, the adaptive setup,
// the multigrid cycle and the Krylov solvers, all driving the kernels of
// fine.cu, transfer.cu, coarse.cu and blas.cu on one stream.
#include "internal.h"
#include "kernels.h"
#include "lqcd_amg.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <array>
#include <vector>

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

using cplx = std::complex<double>;

namespace {

thread_local std::string g_err;

amg_status fail(amg_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

#define CK(x)                                                                                    \
    do {                                                                                         \
        cudaError_t e_ = (x);                                                                    \
        if (e_ != cudaSuccess)                                                                   \
            return fail(AMG_ECUDA, std::string(#x) + " -> " + cudaGetErrorString(e_));          \
    } while (0)
#define TRY(x)                        \
    do {                              \
        amg_status s_ = (x);          \
        if (s_ != AMG_OK) return s_;  \
    } while (0)

int coarse_elem_bytes(int prec) { return prec == 0 ? 16 : 8; }
int vec_prec_of(int fine_prec) { return fine_prec == 0 ? 0 : 1; }

}  // namespace

struct amg_lattice {
    GeomH g;
};
struct amg_gauge {
    amg_lattice* lat;
    DevBuf U[4];   // by precision id: F64, F32, F16, FP64 as float hi/lo pairs
};
struct amg_dirac {
    amg_gauge* gauge;
    double kappa, csw;
    DevBuf C[4];
    DevBuf Ci[3];    // clover inverse A^{-1} by precision (F64, F32, F16), built when an even-odd smoother needs it
    DevBuf in, out;   // call scratch for the canonical-layout entry points
    DevBuf split;     // AMG_F64D: the FP32 parts hi, lo of the input
};

namespace {

struct CoarseLevel {
    GeomH g;
    int nc = 0;
    int prec = 1;        // vector / arithmetic precision: 0 FP64, 1 FP32
    bool opbf = false;   // operator additionally stored in bfloat16 (B16) and applied from there
    bool op32 = false;   // FP64 coarsest level whose Galerkin operator comes from an FP32 level: its
                         // entries are FP32-exact, so B is stored in FP32 and widened in the kernels
    DevBuf B, B16;
    DevBuf tci;                 // bfloat16 stencil in the tensor-core operand layout (multi-RHS apply)
    DevBuf tcx;                 // packed bfloat16 vectors of one tensor-core launch
    DevBuf cs_part, cs_state;   // persistent coarse solver scratch
    // levels between the fine and the coarsest grid: the level's own test
    // vectors (coarsening to the next level) and its FGMRES(inter_m) space
    DevBuf cvecs;
    DevBuf cvecs_next;          // (0-b): the pass's new vectors while M still reads cvecs
    int xgroup = 0;             // coarsest solver's shared-memory tile (coarse sites per gather), tuned
    std::vector<DevBuf> tcw;    // tensor-core coarse solve: r~, R_0..R_l, U_0..U_l (one batch each)
    DevBuf tcerr;
    std::vector<DevBuf> gV, gZ;
    DevBuf gw, gr, gt;
    int kprec() const { return opbf ? 2 : op32 ? 3 : prec; }   // precision code of the stencil kernels
    int bprec() const { return op32 ? 1 : prec; }               // storage precision of B
    const void* op() const { return opbf ? B16.p : B.p; }
};

// pinned partial-sum staging for reductions
struct Reducer {
    DevBuf dpart;
    double2* hpart = nullptr;
    int grid = 0;
    ~Reducer() {
        if (hpart) cudaFreeHost(hpart);
    }
    int cap = 0;
    amg_status init(int nb) {
        grid = blas_grid();
        if (nb <= cap && hpart) return AMG_OK;
        CK(dpart.ensure(sizeof(double2) * grid * 20 * nb));
        if (hpart) cudaFreeHost(hpart);
        hpart = nullptr;
        CK(cudaMallocHost(&hpart, sizeof(double2) * grid * 20 * nb));
        cap = nb;
        return AMG_OK;
    }
    // k dots <a_j, b>
    amg_status dots(int prec, int k, const void* const* a, const void* b, size_t n, cplx* out, cudaStream_t s) {
        CK(launch_multi_dot(prec, k, a, b, n, dpart.as<double2>(), s));
        CK(cudaMemcpyAsync(hpart, dpart.p, sizeof(double2) * grid * k, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int j = 0; j < k; ++j) {
            double re = 0, im = 0;
            for (int q = 0; q < grid; ++q) {
                re += hpart[j * grid + q].x;
                im += hpart[j * grid + q].y;
            }
            out[j] = cplx(re, im);
        }
        return AMG_OK;
    }
    // for r < nb: k dots <a_r[j], b_r> (a_r = a + r * stride entries, likewise b), one
    // synchronisation for the batch; out[r * k + j]; k * nb <= 20 * capacity
    amg_status batch_dots(int prec, int nb, int k, const void* const* a, const void* b, size_t stride, size_t n,
                          cplx* out, cudaStream_t s) {
        const size_t eb = prec == 0 ? 16 : 8;
        std::vector<const void*> ar(k);
        for (int r = 0; r < nb; ++r) {
            for (int j = 0; j < k; ++j) ar[j] = (const char*)a[j] + r * stride * eb;
            CK(launch_multi_dot(prec, k, ar.data(), (const char*)b + r * stride * eb, n,
                                dpart.as<double2>() + (size_t)r * k * grid, s));
        }
        CK(cudaMemcpyAsync(hpart, dpart.p, sizeof(double2) * grid * k * nb, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int j = 0; j < k * nb; ++j) {
            double re = 0, im = 0;
            for (int q = 0; q < grid; ++q) {
                re += hpart[j * grid + q].x;
                im += hpart[j * grid + q].y;
            }
            out[j] = cplx(re, im);
        }
        return AMG_OK;
    }
    amg_status dot(int prec, const void* a, const void* b, size_t n, cplx* out, cudaStream_t s) {
        const void* l[1] = {a};
        return dots(prec, 1, l, b, n, out, s);
    }
    amg_status norm2(int prec, const void* a, size_t n, double* out, cudaStream_t s) {
        CK(launch_norm2(prec, a, n, (double*)dpart.p, s));
        CK(cudaMemcpyAsync(hpart, dpart.p, sizeof(double) * grid, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const double* h = (const double*)hpart;
        double t = 0;
        for (int q = 0; q < grid; ++q) t += h[q];
        *out = t;
        return AMG_OK;
    }
};

inline double2 d2(cplx c) { return make_double2(c.real(), c.imag()); }

// phase timers (Table 1 split: coarse / smoother / R+P / other)
enum Phase { PH_COARSE = 0, PH_SMOOTH = 1, PH_RP = 2, PH_PROD = 3, PH_ORTH = 4, PH_RESID = 5, PH_NPH = 6 };
struct PhaseTimer {
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, int>> marks;   // (event index, phase) start/stop pairs
    std::vector<int> phase_of;
    size_t used = 0;
    bool on = false;
    ~PhaseTimer() {
        for (auto e : pool) cudaEventDestroy(e);
    }
    cudaEvent_t next() {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    void start(int ph, cudaStream_t s) {
        if (!on) return;
        cudaEvent_t e = next();
        cudaEventRecord(e, s);
        phase_of.push_back(ph);
    }
    void stop(cudaStream_t s) {
        if (!on) return;
        cudaEvent_t e = next();
        cudaEventRecord(e, s);
    }
    void reset() {
        used = 0;
        phase_of.clear();
    }
    void collect(double ms[PH_NPH]) {
        for (int i = 0; i < PH_NPH; ++i) ms[i] = 0;
        for (size_t k = 0; k < phase_of.size(); ++k) {
            float t = 0;
            cudaEventSynchronize(pool[2 * k + 1]);
            cudaEventElapsedTime(&t, pool[2 * k], pool[2 * k + 1]);
            ms[phase_of[k]] += t;
        }
    }
};

}  // namespace

struct amg_hierarchy {
    amg_dirac* d = nullptr;
    amg_params p;
    int fp = 1;     // smoother precision used by the solve
    int vp = 1;     // test-vector precision (and the setup's cycle precision)
    int rp = 1;     // precision of the test vectors restriction and prolongation read (vp, or 2 = FP16)
    BlockH blk[AMG_MAX_LEVELS - 1];
    DevBuf vecs0;
    DevBuf vecs16;   // half-precision copy of vecs0 for restriction / prolongation (rp == 2)
    DevBuf vecs_next;   // (0-b): the pass's new vectors while the cycle still reads vecs0 (rp != 2)
    DevBuf tmpg;        // setup: smoothed / cycled outputs of a group of test vectors
    std::vector<CoarseLevel> lev;   // lev[l] for l = 1..nlevels-1 (lev[0] unused)
    // fine workspaces per precision: b, x
    DevBuf fb[3], fx[3];
    // setup scratch
    DevBuf tmpv;
    // coarse workspaces per level: bc, xc, Krylov vectors
    std::vector<std::vector<DevBuf*>> cw;
    // outer FGMRES (FP64 internal fine vectors)
    DevBuf ob, ox, ow, orr;
    std::vector<DevBuf*> oV, oZ;
    DevBuf bv[6], bz[2];   // flexible BiCGStab: r, r~, p, s, t, D M p (FP64); M p, M s (Z precision)
    std::vector<DevBuf> mb;   // MBiCGs inner BiCGStab(l): r~, R_0..R_l, U_0..U_l (smoother precision)
    DevBuf canon;   // canonical staging
    Reducer red;
    // outer Gram-Schmidt with device-side coefficients: per right-hand side three regions of
    // 20 x blas_grid() partials and 64 coefficient slots (pass-1 dots, pass-2 dots at 32, |w| at 63)
    DevBuf gs_part, gs_coef;
    double2* gs_hcoef = nullptr;
    int gs_cap = 0;
    PhaseTimer timer;
    int err_flag_host = 0;
    DevBuf err_flag;
    DevBuf ac_in, ac_out;   // amg_apply_coarse: vectors converted to the level's precision (kept)
    int coarse_cycles = 0;
    int sap_variant[3] = {0, 0, 0};      // chosen SAP kernel per smoother precision, one right-hand side
    int sap_variant_nb[3] = {0, 0, 0};   // the same for batches (the staged kernel then takes two per CTA)
    amg_nn* nn = nullptr;             // learned correction after the cycle (FP32 smoother only)
    bool nn_off = false;              // set while falling back to the plain cycle
    int* hstate = nullptr;   // pinned mirror of the coarse solver state words (16 x 4 ints)
    int tc_cycles = 0;       // coarsest-level cycles of the tensor-core solver in the current solve
    int nb_cap = 0;          // batch width the workspaces are sized for
    // ragged solves: step j of the outer solver (Z_j = M V_j, w = D Z_j) captured as a CUDA graph
    bool graph_mode = false;   // set while capturing: coarse solves run as one cluster
    std::vector<cudaGraphExec_t> gexec;
    std::vector<unsigned long long> gkernels;   // kernels in each captured graph (counted per replay)
    void clear_graphs() {
        for (auto g : gexec)
            if (g) cudaGraphExecDestroy(g);
        gexec.clear();
        gkernels.clear();
    }
    // amg_solve with host vectors: device staging of one batch of canonical b, a copy stream
    // and its events (b staged, b consumed, x staged, x copied out).  x is staged in the last
    // Arnoldi basis vector oV[outer_m] (free between solves, written only at a cycle's last
    // step, which then waits for the copy-out: io_x_pending)
    DevBuf io_b;
    bool io_x_pending = false;
    cudaStream_t io_st = nullptr;
    cudaEvent_t io_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    ~amg_hierarchy() {
        for (auto e : io_ev)
            if (e) cudaEventDestroy(e);
        if (io_st) cudaStreamDestroy(io_st);
        clear_graphs();
        if (hstate) cudaFreeHost(hstate);
        if (gs_hcoef) cudaFreeHost(gs_hcoef);
        for (auto& v : cw)
            for (auto* b : v) delete b;
        for (auto* b : oV) delete b;
        for (auto* b : oZ) delete b;
    }
};

namespace {

const GeomH& fine_geom(amg_hierarchy* h) { return h->d->gauge->lat->g; }
size_t fine_n(amg_hierarchy* h) { return (size_t)fine_geom(h).V * 12; }
size_t coarse_n(const CoarseLevel& L) { return (size_t)L.g.V * L.nc; }
// the test vectors restriction and prolongation read (precision h->rp)
const void* rp_vecs(amg_hierarchy* h) { return h->rp == 2 ? h->vecs16.p : h->vecs0.p; }

amg_status check_params(const GeomH& g, const amg_params* p) {
    if (!p) return fail(AMG_EINVAL, "params is NULL");
    if (p->nlevels < 2 || p->nlevels > AMG_MAX_LEVELS) return fail(AMG_EINVAL, "nlevels must be 2..4");
    int L[4] = {g.L[0], g.L[1], g.L[2], g.L[3]};
    for (int l = 0; l < p->nlevels - 1; ++l) {
        if (p->nvec[l] < 1 || p->nvec[l] > 64) return fail(AMG_EINVAL, "nvec must be in 1..64");
        for (int mu = 0; mu < 4; ++mu) {
            int b = p->block[l][mu];
            if (b < 1 || L[mu] % b != 0) return fail(AMG_EINVAL, "block does not tile the lattice");
            int C = L[mu] / b;
            if (C < 2 || C % 2 != 0)
                return fail(AMG_EINVAL, "need an even number (>= 2) of blocks per direction (SAP colouring)");
            L[mu] = C;
        }
        int vb = p->block[l][0] * p->block[l][1] * p->block[l][2] * p->block[l][3];
        if (vb > 512) return fail(AMG_EINVAL, "block volume must be <= 512 sites");
        if (l >= 1) {
            // coarse-level Galerkin kernel: Nc_next = 2 nvec <= 64 and its shared-memory tiles
            const int nc = 2 * p->nvec[l - 1], nv = p->nvec[l];
            const size_t esz = p->prec_coarse == AMG_F64 ? 16 : 8;
            if (nv > 32) return fail(AMG_EINVAL, "nvec of a coarse level must be <= 32");
            if ((size_t)(4 * nc * nv + nc * nc) * esz > 200 * 1024)
                return fail(AMG_EINVAL, "coarse level too wide for the Galerkin kernel's shared memory");
        }
    }
    if (p->nlevels >= 3) {
        if (p->prec_coarse != AMG_F64 && p->prec_coarse != AMG_F32 && p->prec_coarse != AMG_BF16)
            return fail(AMG_EINVAL, "prec_coarse must be AMG_F64, AMG_F32 or AMG_BF16");
        if (p->prec_coarse == AMG_F64 && p->prec_coarsest != AMG_F64)
            return fail(AMG_EINVAL, "an FP64 intermediate level needs an FP64 coarsest level");
        if (p->inter_m < 1 || p->inter_m > 19 || p->inter_maxit < 1 || !(p->inter_tol > 0))
            return fail(AMG_EINVAL, "inter_m must be 1..19, inter_maxit >= 1, inter_tol > 0");
    }
    if (p->prec_smoother < 0 || p->prec_smoother > 2) return fail(AMG_EINVAL, "prec_smoother");
    if (p->prec_coarsest != AMG_F64 && p->prec_coarsest != AMG_F32 && p->prec_coarsest != AMG_BF16)
        return fail(AMG_EINVAL, "prec_coarsest must be AMG_F64, AMG_F32 or AMG_BF16");
    // the coarse solver streams operator rows with bulk copies that need 16-byte multiples:
    // 9 * Nc bfloat16 pairs per row, so Nc = 2 nvec must be a multiple of 4
    if (p->prec_coarsest == AMG_BF16 && p->nvec[p->nlevels - 2] % 2 != 0)
        return fail(AMG_EINVAL, "a bfloat16 coarsest operator needs an even number of test vectors");
    if (p->coarse_ell < 1 || p->coarse_ell > 4) return fail(AMG_EINVAL, "coarse_ell must be 1..4");
    if (p->outer_m < 1 || p->outer_m > 19) return fail(AMG_EINVAL, "outer_m must be 1..19");
    if (p->outer_solver < 0 || p->outer_solver > 2) return fail(AMG_EINVAL, "outer_solver must be 0, 1 or 2");
    if (p->sap_variant < -1 || p->sap_variant > 3) return fail(AMG_EINVAL, "sap_variant must be -1, 0, 1, 2 or 3");
    if (p->resid_pair != 0 && p->resid_pair != 1) return fail(AMG_EINVAL, "resid_pair must be 0 or 1");
    if (p->sap_eo != 0 && p->sap_eo != 1) return fail(AMG_EINVAL, "sap_eo must be 0 or 1");
    if (p->sap_eo) {
        BlockH b0;
        for (int mu = 0; mu < 4; ++mu) b0.b[mu] = p->block[0][mu];
        if (!sap_eo_supported(b0))
            return fail(AMG_EINVAL, "even-odd SAP needs an even block extent in x and at most 512 sites per block");
    }
    if (p->outer_solver == 2 && p->prec_smoother == AMG_F16)
        return fail(AMG_EINVAL, "MBiCGs (outer_solver 2) runs its inner BiCGStab in FP32 or FP64");
    if (p->outer_solver == 2 && (!(p->mbicgs_tol > 0) || p->mbicgs_maxit < 1))
        return fail(AMG_EINVAL, "MBiCGs needs mbicgs_tol > 0 and mbicgs_maxit >= 1");
    if (p->prec_vectors == AMG_F16 && p->prec_smoother == AMG_F64)
        return fail(AMG_EINVAL, "half-precision test vectors need an FP32 or FP16 smoother");
    if (p->sap_iters < 0 || p->mr_iters < 0) return fail(AMG_EINVAL, "sap_iters / mr_iters");
    return AMG_OK;
}

// ---------------------------------------------------------------- fine ops
// Every operation below works on a batch of nb right-hand sides stored one
// after another (field q at byte offset q * field size).
size_t fsz(amg_hierarchy* h, int prec) { return fine_spinor_bytes(prec, fine_geom(h).V); }
void* fld(const DevBuf& b, amg_hierarchy* h, int prec, int q) { return (char*)b.p + q * fsz(h, prec); }

amg_status fine_D(amg_hierarchy* h, int prec, const void* in, void* out, const void* b, int nb, cudaStream_t s) {
    amg_dirac* d = h->d;
    CK(launch_dirac(prec, fine_geom(h), nullptr, d->gauge->U[prec].p, d->C[prec].p, in, out, b, d->kappa, nb, s));
    return AMG_OK;
}

// r = b - D x for FP64 internal x and b (the outer solver's true residual, reading C29): the
// double-float stencil where the FP64-valued link and clover pairs exist (FP32 smoother),
// else the FP64 stencil
amg_status true_residual(amg_hierarchy* h, const void* x, void* r, const void* b, int nb, cudaStream_t s) {
    amg_dirac* d = h->d;
    if (h->p.resid_pair && h->fp != 0 && d->gauge->U[3].p && d->C[3].p && d->gauge->U[1].p && d->C[1].p) {
        // x split into the FP32 workspaces (free between cycles; nb fields each when fp != 0)
        CK(launch_dirac_dd(fine_geom(h), d->gauge->U[3].p, d->C[3].p, d->gauge->U[1].p, d->C[1].p, x, r, b,
                           d->kappa, nb, h->fb[1].p, h->fx[1].p, s));
        return AMG_OK;
    }
    return fine_D(h, 0, x, r, b, nb, s);
}

// one SAP half sweep with kernel variant var (0-2: launch_sap_half_variant; 3: FP32 vectors
// with the domain operator staged from its FP16 copy)
cudaError_t sap_half_launch(amg_dirac* d, int var, int prec, const GeomH& g, const BlockH& bk, int colour, int nmr,
                            int x_mode, const void* b, void* x, int nb, cudaStream_t s) {
    if (var == 3 && prec == 1)
        return launch_sap_half_staged16(g, bk, colour, nmr, x_mode, d->gauge->U[1].p, d->C[1].p, d->gauge->U[2].p,
                                        d->C[2].p, b, x, d->kappa, nb, s);
    return launch_sap_half_variant(var == 3 ? 1 : var, prec, g, bk, colour, nmr, x_mode, d->gauge->U[prec].p,
                                   d->C[prec].p, b, x, d->kappa, nb, s);
}

amg_status fine_sap(amg_hierarchy* h, int prec, const void* b, void* x, bool x_zero, int nb, cudaStream_t s) {
    amg_dirac* d = h->d;
    h->timer.start(PH_SMOOTH, s);
    const int var = nb > 1 ? h->sap_variant_nb[prec] : h->sap_variant[prec];
    for (int i = 0; i < h->p.sap_iters; ++i) {
        const bool first = x_zero && i == 0;
        for (int colour = 0; colour < 2; ++colour) {
            const int x_mode = first ? (colour == 0 ? 1 : 2) : 0;
            if (h->p.sap_eo)
                CK(launch_sap_half_eo(prec, fine_geom(h), h->blk[0], colour, h->p.mr_iters, x_mode,
                                      d->gauge->U[prec].p, d->C[prec].p, d->Ci[prec].p, b, x, d->kappa, nb, s));
            else
                CK(sap_half_launch(d, var, prec, fine_geom(h), h->blk[0], colour, h->p.mr_iters, x_mode, b, x, nb,
                                   s));
        }
    }
    if (h->p.sap_iters == 0 && x_zero) CK(cudaMemsetAsync(x, 0, fsz(h, prec) * nb, s));
    h->timer.stop(s);
    return AMG_OK;
}

// ---------------------------------------------------------------- coarse solve
CoarseLevel& L1(amg_hierarchy* h) { return h->lev[1]; }

// BiCGStab(l) (Sleijpen-Fokkema) on the coarsest level to relative tolerance
// coarse_tol: one persistent cooperative launch per group of up to
// coarse_solver_max_rhs() right-hand sides in lockstep (the operator streamed
// once per stencil pass for the group), no host synchronisation.
amg_status coarse_bicgstab_tc(amg_hierarchy* h, int l, const void* b, void* x, int nb, cudaStream_t s);
bool bicgstab_mr_coefficients(const std::vector<std::vector<cplx>>& G, int ell, std::vector<cplx>& cxv,
                              std::vector<cplx>& crv, std::vector<cplx>& cgv);
amg_status coarse_bicgstab(amg_hierarchy* h, int l, const void* b, void* x, int nb, cudaStream_t s) {
    CoarseLevel& L = h->lev[l];
    // batches on a bfloat16 coarsest level: the stencil passes on the tensor cores
    if (h->p.coarse_tc && nb >= 2 && !h->graph_mode && L.opbf && L.prec == 1 && coarse_tc_supported(L.nc) &&
        nb <= 16 && L.tci.p)
        return coarse_bicgstab_tc(h, l, b, x, nb, s);
    const int ell = h->p.coarse_ell;
    auto& w = h->cw[l];   // [0] bc, [1] xc (nb vectors each), [2] rt, [3..3+ell] R, [4+ell..4+2ell] U
    void* R[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    void* U[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int j = 0; j <= ell; ++j) {
        R[j] = w[3 + j]->p;
        U[j] = w[4 + ell + j]->p;
    }
    const size_t cv = coarse_n(L) * coarse_elem_bytes(L.prec);
    const int group = h->graph_mode ? 1 : coarse_solver_max_rhs();
    for (int q = 0, k = 0; q < nb; q += group, ++k) {
        const int ng = std::min(group, nb - q);
        CK(cudaMemsetAsync(L.cs_state.p, 0, 12, s));
        CK(launch_coarse_bicgstab(L.kprec(), L.g, L.nc, L.op(), (const char*)b + q * cv, (char*)x + q * cv, w[2]->p, R,
                                  U, ell, h->p.coarse_tol, h->p.coarse_maxit, L.cs_part.p, L.cs_state.p,
                                  h->graph_mode ? 8 : 0, s, ng, L.xgroup));
        // error word of this launch (a later one would overwrite it): fold into word 2 of the host mirror
        CK(cudaMemcpyAsync(h->hstate + 4 * (k % 16), L.cs_state.p, 16, cudaMemcpyDeviceToHost, s));
    }
    return AMG_OK;
}

// BiCGStab(l) (Sleijpen-Fokkema) in lockstep over a batch of nb right-hand sides on a
// coarsest level stored in bfloat16, every stencil pass on the tensor cores: one
// launch_coarse_apply_tc for the whole batch (bfloat16 operands, FP32 accumulation in tensor
// memory).  The vector updates run on the FP32 pipe, the per-RHS scalars on the host (one
// synchronisation per reduction for the batch); each right-hand side keeps its own scalars and
// stopping test and is frozen once it has converged.  The MMA rounds the vectors to bfloat16
// (reading C18), so the recursive residual drifts from the true one by ~1e-3: the coarse
// tolerance of 1e-2 stays reachable.
amg_status coarse_bicgstab_tc(amg_hierarchy* h, int l, const void* b, void* x, int nb, cudaStream_t s) {
    CoarseLevel& L = h->lev[l];
    const int ell = h->p.coarse_ell;
    const size_t n = coarse_n(L), vb = n * sizeof(float2);
    while ((int)L.tcw.size() < 2 * ell + 3) L.tcw.emplace_back();
    for (auto& v : L.tcw) CK(v.ensure(vb * nb));
    CK(L.tcx.ensure(coarse_tc_pack_bytes(L.g.V, L.nc)));
    CK(L.tcerr.ensure(sizeof(int)));
    CK(cudaMemsetAsync(L.tcerr.p, 0, sizeof(int), s));
    void* rt = L.tcw[0].p;
    std::vector<void*> R(ell + 1), U(ell + 1);
    for (int j = 0; j <= ell; ++j) {
        R[j] = L.tcw[1 + j].p;
        U[j] = L.tcw[2 + ell + j].p;
    }
    auto F = [&](const void* base, int r) { return (char*)base + r * vb; };
    const double2 one = make_double2(1, 0);
    Reducer& red = h->red;
    TRY(red.init(std::max(nb, 2)));
    CK(cudaMemsetAsync(x, 0, vb * nb, s));
    CK(cudaMemsetAsync(U[0], 0, vb * nb, s));
    CK(cudaMemcpyAsync(R[0], b, vb * nb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(rt, b, vb * nb, cudaMemcpyDeviceToDevice, s));
    std::vector<cplx> rho0(nb, 1.0), rho1(nb, 0.0), alpha(nb, 0.0), omega(nb, 1.0);
    std::vector<double> bn2(nb, -1.0);
    std::vector<char> act(nb, 1);
    auto stencil = [&](const void* in, void* out) -> amg_status {
        CK(launch_coarse_apply_tc(L.g, L.nc, L.tci.p, in, out, nullptr, nb, L.tcx.p, L.tcerr.as<int>(), s));
        return AMG_OK;
    };
    int cycle = 0;
    for (;; ++cycle) {
        // |R_0|^2 and <r~, R_0> per right-hand side
        std::vector<cplx> q(2 * nb);
        {
            const void* a2[2] = {R[0], rt};
            TRY(red.batch_dots(1, nb, 2, a2, R[0], n, n, q.data(), s));
        }
        bool any = false;
        for (int r = 0; r < nb; ++r) {
            if (!act[r]) continue;
            const double rn2 = q[2 * r].real();
            if (bn2[r] < 0) bn2[r] = rn2;
            if (!std::isfinite(rn2)) return fail(AMG_NAN, "coarse solver: non-finite residual");
            if (rn2 <= h->p.coarse_tol * h->p.coarse_tol * bn2[r] || cycle >= h->p.coarse_maxit) {
                act[r] = 0;
                continue;
            }
            any = true;
            rho1[r] = q[2 * r + 1];
            rho0[r] = -omega[r] * rho0[r];
        }
        if (!any) break;
        for (int j = 0; j < ell; ++j) {
            for (int r = 0; r < nb; ++r) {
                if (!act[r]) continue;
                const cplx beta = alpha[r] * rho1[r] / rho0[r];
                rho0[r] = rho1[r];
                for (int i = 0; i <= j; ++i) CK(launch_axpby(1, one, F(R[i], r), d2(-beta), F(U[i], r), n, s));
            }
            TRY(stencil(U[j], U[j + 1]));
            std::vector<cplx> gam(nb);
            {
                const void* a1[1] = {rt};
                TRY(red.batch_dots(1, nb, 1, a1, U[j + 1], n, n, gam.data(), s));
            }
            for (int r = 0; r < nb; ++r) {
                if (!act[r]) continue;
                alpha[r] = rho0[r] / gam[r];
                if (!std::isfinite(alpha[r].real()) || !std::isfinite(alpha[r].imag()))
                    return fail(AMG_NAN, "coarse solver: BiCGStab breakdown");
                for (int i = 0; i <= j; ++i) CK(launch_axpby(1, d2(-alpha[r]), F(U[i + 1], r), one, F(R[i], r), n, s));
                CK(launch_axpby(1, d2(alpha[r]), F(U[0], r), one, F(x, r), n, s));
            }
            TRY(stencil(R[j], R[j + 1]));
            if (j + 1 < ell) {
                std::vector<cplx> r1(nb);
                const void* a1[1] = {rt};
                TRY(red.batch_dots(1, nb, 1, a1, R[j + 1], n, n, r1.data(), s));
                for (int r = 0; r < nb; ++r)
                    if (act[r]) rho1[r] = r1[r];
            }
        }
        // Gram matrices G_pq = <R_p, R_q> of every right-hand side, then the minimal-residual part
        std::vector<cplx> gm((size_t)nb * (ell + 1) * (ell + 1));
        for (int qq = 0; qq <= ell; ++qq) {
            std::vector<cplx> row((size_t)nb * (ell + 1));
            std::vector<const void*> al(R.begin(), R.end());
            TRY(red.batch_dots(1, nb, ell + 1, al.data(), R[qq], n, n, row.data(), s));
            for (int r = 0; r < nb; ++r)
                for (int p = 0; p <= ell; ++p) gm[((size_t)r * (ell + 1) + p) * (ell + 1) + qq] = row[r * (ell + 1) + p];
        }
        for (int r = 0; r < nb; ++r) {
            if (!act[r]) continue;
            std::vector<std::vector<cplx>> G(ell + 1, std::vector<cplx>(ell + 1));
            for (int p = 0; p <= ell; ++p)
                for (int qq = 0; qq <= ell; ++qq) G[p][qq] = gm[((size_t)r * (ell + 1) + p) * (ell + 1) + qq];
            std::vector<cplx> cxv, crv, cgv;
            if (!bicgstab_mr_coefficients(G, ell, cxv, crv, cgv))
                return fail(AMG_NAN, "coarse solver: BiCGStab breakdown");
            omega[r] = cgv[ell];
            CK(launch_axpby(1, d2(cxv[0]), F(R[0], r), one, F(x, r), n, s));
            for (int k = 1; k <= ell; ++k) {
                CK(launch_axpby(1, d2(cxv[k]), F(R[k], r), one, F(x, r), n, s));
                CK(launch_axpby(1, d2(-crv[k]), F(R[k], r), one, F(R[0], r), n, s));
                CK(launch_axpby(1, d2(-cgv[k]), F(U[k], r), one, F(U[0], r), n, s));
            }
        }
    }
    int terr = 0;
    CK(cudaMemcpyAsync(&terr, L.tcerr.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (terr) return fail(AMG_TIMEOUT, "tensor-core coarse stencil: a bounded wait gave up");
    h->tc_cycles += cycle;
    return AMG_OK;
}

// status of the last batch of coarse solves; valid after any stream synchronisation
amg_status coarse_status(amg_hierarchy* h) {
    for (int q = 0; q < 16; ++q) {
        if (h->hstate[4 * q + 2] == 1) return fail(AMG_TIMEOUT, "coarse solver: grid barrier timed out");
        if (h->hstate[4 * q + 2] != 0) return fail(AMG_NAN, "coarse solver: breakdown or non-finite residual");
    }
    return AMG_OK;
}

// ---------------------------------------------------------------- levels >= 1 of three or more grids
amg_status coarse_solve(amg_hierarchy* h, int l, const void* b, void* x, int nb, cudaStream_t s);

size_t cvec_bytes(const CoarseLevel& L) { return coarse_n(L) * coarse_elem_bytes(L.prec); }

// SAP (Sec. 3 listing) on level l, started from x (or from zero), right-hand side b
amg_status coarse_sap(amg_hierarchy* h, int l, const void* b, void* x, bool x_zero, int nb, cudaStream_t s) {
    CoarseLevel& L = h->lev[l];
    for (int i = 0; i < h->p.sap_iters; ++i) {
        const bool first = x_zero && i == 0;
        CK(launch_coarse_sap_half(L.kprec(), L.g, h->blk[l], L.nc, 0, h->p.mr_iters, first ? 1 : 0, L.op(), b, x,
                                  nb, s));
        CK(launch_coarse_sap_half(L.kprec(), L.g, h->blk[l], L.nc, 1, h->p.mr_iters, first ? 2 : 0, L.op(), b, x,
                                  nb, s));
    }
    if (h->p.sap_iters == 0 && x_zero) CK(cudaMemsetAsync(x, 0, cvec_bytes(L) * nb, s));
    return AMG_OK;
}

// x = M_l b on level l >= 1: steps (1) and (2) of Sec. 3 one level down.  When
// the next level solves in FP64 while this one works in FP32, the restricted
// vector is widened before the solve and the solution narrowed after it
// (through the next level's shadow vector, free outside its solve).
amg_status vcycle_c(amg_hierarchy* h, int l, const void* b, void* x, cudaStream_t s) {
    CoarseLevel& L = h->lev[l];
    CoarseLevel& N = h->lev[l + 1];
    auto& w = h->cw[l + 1];
    const bool widen = N.prec != L.prec;
    void* rc = widen ? w[2]->p : w[0]->p;
    CK(launch_restrict_coarse(L.prec, L.g, h->blk[l], L.nc, h->p.nvec[l], L.cvecs.p, b, rc, 1, s));
    if (widen) CK(launch_convert_flat(L.prec, N.prec, rc, w[0]->p, coarse_n(N), s));
    TRY(coarse_solve(h, l + 1, w[0]->p, w[1]->p, 1, s));
    if (widen) CK(launch_convert_flat(N.prec, L.prec, w[1]->p, rc, coarse_n(N), s));
    CK(launch_prolong_coarse(L.prec, L.g, h->blk[l], L.nc, h->p.nvec[l], L.cvecs.p, widen ? rc : w[1]->p, x, 1, s));
    return coarse_sap(h, l, b, x, false, 1, s);
}

// one Givens step of the least-squares update of a flexible GMRES column j
void givens_column(std::vector<std::vector<cplx>>& H, std::vector<double>& cs, std::vector<cplx>& sn,
                   std::vector<cplx>& g, int j) {
    for (int i = 0; i < j; ++i) {
        cplx a = H[i][j], bb = H[i + 1][j];
        H[i][j] = cs[i] * a + sn[i] * bb;
        H[i + 1][j] = -std::conj(sn[i]) * a + cs[i] * bb;
    }
    cplx a = H[j][j], bb = H[j + 1][j];
    double aa = std::abs(a), ab = std::abs(bb);
    if (ab == 0) {
        cs[j] = 1;
        sn[j] = 0;
    } else if (aa == 0) {
        cs[j] = 0;
        sn[j] = std::conj(bb) / ab;
    } else {
        double t = std::sqrt(aa * aa + ab * ab);
        cs[j] = aa / t;
        sn[j] = (a / aa) * std::conj(bb) / t;
    }
    H[j][j] = cs[j] * a + sn[j] * bb;
    H[j + 1][j] = 0;
    g[j + 1] = -std::conj(sn[j]) * g[j];
    g[j] = cs[j] * g[j];
}

// Flexible GMRES(inter_m) on an intermediate level l, preconditioned by the
// level's own cycle, from x = 0 until the residual is below inter_tol |b| or
// inter_maxit steps were taken; the true residual b - D_l x is recomputed
// after every cycle (reading C12).  Vectors in the level's precision,
// reductions in FP64.
amg_status fgmres_c(amg_hierarchy* h, int l, const void* b, void* x, cudaStream_t s) {
    CoarseLevel& L = h->lev[l];
    const int m = h->p.inter_m, pr = L.prec;
    const size_t n = coarse_n(L), vb = cvec_bytes(L);
    const double tol = h->p.inter_tol;
    Reducer& red = h->red;
    CK(cudaMemsetAsync(x, 0, vb, s));
    double bn2;
    TRY(red.norm2(pr, b, n, &bn2, s));
    TRY(coarse_status(h));
    if (!std::isfinite(bn2)) return fail(AMG_NAN, "intermediate solve: non-finite right-hand side");
    const double bn = std::sqrt(bn2);
    if (bn == 0) return AMG_OK;
    int iters = 0;
    bool first = true;
    std::vector<std::vector<cplx>> H(m + 1, std::vector<cplx>(m));
    std::vector<double> cs(m);
    std::vector<cplx> sn(m), g(m + 1);
    while (true) {
        double rn;
        if (first) {   // x = 0: r = b
            CK(cudaMemcpyAsync(L.gr.p, b, vb, cudaMemcpyDeviceToDevice, s));
            rn = bn;
            first = false;
        } else {
            CK(launch_coarse_apply(L.kprec(), L.g, L.nc, nullptr, L.op(), x, L.gr.p, b, 1, s));
            double rn2;
            TRY(red.norm2(pr, L.gr.p, n, &rn2, s));
            TRY(coarse_status(h));
            if (!std::isfinite(rn2)) return fail(AMG_NAN, "intermediate solve: non-finite residual");
            rn = std::sqrt(rn2);
        }
        if (rn <= tol * bn || iters >= h->p.inter_maxit) return AMG_OK;
        for (auto& row : H) std::fill(row.begin(), row.end(), cplx(0));
        std::fill(g.begin(), g.end(), cplx(0));
        g[0] = rn;
        CK(launch_axpby(pr, make_double2(1.0 / rn, 0), L.gr.p, make_double2(0, 0), L.gV[0].p, n, s));
        int jend = -1;
        for (int j = 0; j < m; ++j) {
            TRY(vcycle_c(h, l, L.gV[j].p, L.gZ[j].p, s));
            CK(launch_coarse_apply(L.kprec(), L.g, L.nc, nullptr, L.op(), L.gZ[j].p, L.gw.p, nullptr, 1, s));
            std::vector<const void*> vl(j + 1);
            for (int i = 0; i <= j; ++i) vl[i] = L.gV[i].p;
            std::vector<cplx> c(j + 1);
            std::vector<double2> nc(j + 1);
            for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
                TRY(red.dots(pr, j + 1, vl.data(), L.gw.p, n, c.data(), s));
                if (pass == 0) TRY(coarse_status(h));
                for (int i = 0; i <= j; ++i) {
                    H[i][j] += c[i];
                    nc[i] = make_double2(-c[i].real(), -c[i].imag());
                }
                CK(launch_multi_axpy(pr, j + 1, nc.data(), vl.data(), L.gw.p, n, s));
            }
            double hn2;
            TRY(red.norm2(pr, L.gw.p, n, &hn2, s));
            const double hn = std::sqrt(hn2);
            H[j + 1][j] = hn;
            ++iters;
            givens_column(H, cs, sn, g, j);
            jend = j;
            const double est = std::abs(g[j + 1]);
            if (!std::isfinite(est)) return fail(AMG_NAN, "intermediate solve: non-finite Arnoldi coefficient");
            if (hn == 0 || est <= tol * bn || iters >= h->p.inter_maxit) break;
            CK(launch_axpby(pr, make_double2(1.0 / hn, 0), L.gw.p, make_double2(0, 0), L.gV[j + 1].p, n, s));
        }
        const int k = jend + 1;
        std::vector<cplx> y(k);
        for (int i = k - 1; i >= 0; --i) {
            cplx t = g[i];
            for (int c = i + 1; c < k; ++c) t -= H[i][c] * y[c];
            y[i] = t / H[i][i];
        }
        std::vector<double2> yc(k);
        std::vector<const void*> zl(k);
        for (int i = 0; i < k; ++i) {
            yc[i] = d2(y[i]);
            zl[i] = L.gZ[i].p;
        }
        CK(launch_multi_axpy(pr, k, yc.data(), zl.data(), x, n, s));
    }
}

// loose solve on level l: BiCGStab(ell) on the coarsest level, else the
// level's flexible GMRES (one right-hand side at a time)
amg_status coarse_solve(amg_hierarchy* h, int l, const void* b, void* x, int nb, cudaStream_t s) {
    if (l == h->p.nlevels - 1) return coarse_bicgstab(h, l, b, x, nb, s);
    const size_t vb = cvec_bytes(h->lev[l]);
    for (int q = 0; q < nb; ++q) TRY(fgmres_c(h, l, (const char*)b + q * vb, (char*)x + q * vb, s));
    return AMG_OK;
}

// ---------------------------------------------------------------- V-cycle
// x = M b on the fine lattice in precision prec (b, x internal fields, nb of them):
// step (1) x = P D_c^{-1} R b, step (2) x += SAP(b - D x).
amg_status vcycle0(amg_hierarchy* h, int prec, const void* b, void* x, int nb, cudaStream_t s) {
    CoarseLevel& L = L1(h);
    auto& w = h->cw[1];
    h->timer.start(PH_RP, s);
    CK(launch_restrict_fine(prec, h->rp, L.prec, fine_geom(h), h->blk[0], h->p.nvec[0], rp_vecs(h), b, w[0]->p, nb,
                            s));
    h->timer.stop(s);
    h->timer.start(PH_COARSE, s);
    TRY(coarse_solve(h, 1, w[0]->p, w[1]->p, nb, s));
    h->timer.stop(s);
    h->timer.start(PH_RP, s);
    CK(launch_prolong_fine(prec, h->rp, L.prec, fine_geom(h), h->blk[0], h->p.nvec[0], rp_vecs(h), w[1]->p, x, nb,
                           s));
    h->timer.stop(s);
    TRY(fine_sap(h, prec, b, x, false, nb, s));
    return AMG_OK;
}

// ---------------------------------------------------------------- MBiCGs preconditioner
// Coefficients of the minimal-residual part of BiCGStab(l) from the Gram
// matrix G_pq = <R_p, R_q> (p, q = 0..l): Gram-Schmidt of R_1..R_l in the
// original basis (Rt_j = sum_k C[j][k] R_k, tau_ij = <Rt_i, Rt_j> / sigma_i),
// then x += cx_0 R_0 + sum_k cx_k R_k, R_0 -= sum_k cr_k R_k,
// U_0 -= sum_k cg_k U_k (the same algebra as the coarse solver's kernel).
bool bicgstab_mr_coefficients(const std::vector<std::vector<cplx>>& G, int ell, std::vector<cplx>& cxv,
                              std::vector<cplx>& crv, std::vector<cplx>& cgv) {
    std::vector<std::vector<cplx>> C(ell + 1, std::vector<cplx>(ell + 1, cplx(0))),
        tau(ell + 1, std::vector<cplx>(ell + 1, cplx(0)));
    std::vector<double> sigma(ell + 1, 0.0);
    std::vector<cplx> gp(ell + 1, cplx(0)), g(ell + 1, cplx(0)), gpp(ell + 1, cplx(0));
    for (int j = 1; j <= ell; ++j) {
        C[j][j] = 1;
        for (int i = 1; i < j; ++i) {
            cplx t = 0;
            for (int p = 1; p <= i; ++p)
                for (int q = 1; q <= j; ++q) t += std::conj(C[i][p]) * C[j][q] * G[p][q];
            tau[i][j] = t / sigma[i];
            for (int k = 1; k <= i; ++k) C[j][k] -= tau[i][j] * C[i][k];
        }
        double sg = 0;
        cplx t0 = 0;
        for (int p = 1; p <= j; ++p) {
            for (int q = 1; q <= j; ++q) sg += (std::conj(C[j][p]) * C[j][q] * G[p][q]).real();
            t0 += std::conj(C[j][p]) * G[p][0];
        }
        if (!(sg > 0)) return false;
        sigma[j] = sg;
        gp[j] = t0 / sg;
    }
    g[ell] = gp[ell];
    for (int j = ell - 1; j >= 1; --j) {
        cplx t = gp[j];
        for (int i = j + 1; i <= ell; ++i) t -= tau[j][i] * g[i];
        g[j] = t;
    }
    for (int j = 1; j < ell; ++j) {
        cplx t = g[j + 1];
        for (int i = j + 1; i < ell; ++i) t += tau[j][i] * g[i + 1];
        gpp[j] = t;
    }
    cxv.assign(ell + 1, cplx(0));
    crv.assign(ell + 1, cplx(0));
    cgv = g;
    cxv[0] = g[1];
    for (int j = 1; j < ell; ++j)
        for (int k = 1; k <= j; ++k) cxv[k] += gpp[j] * C[j][k];
    for (int j = 1; j <= ell; ++j)
        for (int k = 1; k <= j; ++k) crv[k] += gp[j] * C[j][k];
    return true;
}

// x = BiCGStab(l)(D, b) on the fine lattice in precision prec (internal fields), from x = 0
// to relative residual mbicgs_tol or mbicgs_maxit cycles: the preconditioner of the paper's
// mixed-precision BiCGStab comparison solver (Sec. 5; reading C27).  Host-driven: every
// cycle is 2l fine stencil passes, whose cost dwarfs the host synchronisations.
amg_status fine_bicgstab_l(amg_hierarchy* h, int prec, const void* b, void* x, cudaStream_t s) {
    const int ell = h->p.coarse_ell;
    const size_t n = fine_n(h), fb = fsz(h, prec);
    Reducer& red = h->red;
    while ((int)h->mb.size() < 2 * ell + 3) h->mb.emplace_back();
    for (auto& v : h->mb) CK(v.ensure(fb));
    void* rt = h->mb[0].p;
    std::vector<void*> R(ell + 1), U(ell + 1);
    for (int j = 0; j <= ell; ++j) {
        R[j] = h->mb[1 + j].p;
        U[j] = h->mb[2 + ell + j].p;
    }
    const double2 one = make_double2(1, 0);
    auto axpy = [&](cplx a, const void* xv, void* yv) -> amg_status {   // y += a x
        CK(launch_axpby(prec, d2(a), xv, one, yv, n, s));
        return AMG_OK;
    };
    CK(cudaMemsetAsync(x, 0, fb, s));
    CK(cudaMemsetAsync(U[0], 0, fb, s));
    CK(cudaMemcpyAsync(R[0], b, fb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(rt, b, fb, cudaMemcpyDeviceToDevice, s));
    double bn2;
    TRY(red.norm2(prec, b, n, &bn2, s));
    if (!std::isfinite(bn2)) return fail(AMG_NAN, "MBiCGs: non-finite right-hand side");
    if (bn2 == 0) return AMG_OK;
    cplx rho0 = 1, alpha = 0, omega = 1;
    const double tol2 = h->p.mbicgs_tol * h->p.mbicgs_tol * bn2;
    for (int cycle = 0; cycle < h->p.mbicgs_maxit; ++cycle) {
        double rn2;
        TRY(red.norm2(prec, R[0], n, &rn2, s));
        if (!std::isfinite(rn2)) return fail(AMG_NAN, "MBiCGs: non-finite inner residual");
        if (rn2 <= tol2) break;
        rho0 = -omega * rho0;
        for (int j = 0; j < ell; ++j) {
            cplx rho1;
            TRY(red.dot(prec, rt, R[j], n, &rho1, s));
            const cplx beta = alpha * rho1 / rho0;
            rho0 = rho1;
            for (int i = 0; i <= j; ++i) CK(launch_axpby(prec, one, R[i], d2(-beta), U[i], n, s));   // U_i = R_i - beta U_i
            TRY(fine_D(h, prec, U[j], U[j + 1], nullptr, 1, s));
            cplx gam;
            TRY(red.dot(prec, rt, U[j + 1], n, &gam, s));
            alpha = rho0 / gam;
            if (!std::isfinite(alpha.real()) || !std::isfinite(alpha.imag()))
                return fail(AMG_NAN, "MBiCGs: inner BiCGStab breakdown");
            for (int i = 0; i <= j; ++i) TRY(axpy(-alpha, U[i + 1], R[i]));
            TRY(fine_D(h, prec, R[j], R[j + 1], nullptr, 1, s));
            TRY(axpy(alpha, U[0], x));
        }
        // Gram matrix of R_0..R_l, one row of dots per R_q
        std::vector<std::vector<cplx>> G(ell + 1, std::vector<cplx>(ell + 1));
        std::vector<const void*> Rl(R.begin(), R.end());
        for (int q = 0; q <= ell; ++q) {
            std::vector<cplx> row(ell + 1);
            TRY(red.dots(prec, ell + 1, Rl.data(), R[q], n, row.data(), s));
            for (int p = 0; p <= ell; ++p) G[p][q] = row[p];
        }
        std::vector<cplx> cxv, crv, cgv;
        if (!bicgstab_mr_coefficients(G, ell, cxv, crv, cgv)) return fail(AMG_NAN, "MBiCGs: inner BiCGStab breakdown");
        omega = cgv[ell];
        TRY(axpy(cxv[0], R[0], x));
        for (int k = 1; k <= ell; ++k) {
            TRY(axpy(cxv[k], R[k], x));
            TRY(axpy(-crv[k], R[k], R[0]));
            TRY(axpy(-cgv[k], U[k], U[0]));
        }
    }
    return AMG_OK;
}

// z = M v for FP64 internal fields v; z is written in the outer solver's Z
// precision (FP64 for the all-FP64 path, else FP32: the cycle's output is
// exact in FP32, so nothing is lost).  With outer_solver 2 (MBiCGs) M is the
// inner BiCGStab(l) on the fine operator instead of the multigrid cycle.
int zprec_of(amg_hierarchy* h) { return h->fp == 0 ? 0 : 1; }
amg_status precondition64(amg_hierarchy* h, const void* v, void* z, int nb, cudaStream_t s) {
    const GeomH& g = fine_geom(h);
    int fp = h->fp;
    if (h->p.outer_solver == 2) {
        if (nb != 1) return fail(AMG_EINVAL, "MBiCGs preconditions one right-hand side at a time");
        h->timer.start(PH_SMOOTH, s);
        amg_status st;
        if (fp == 0) {
            st = fine_bicgstab_l(h, 0, v, z, s);
        } else {
            CK(launch_convert_spinor(0, 1, g, v, h->fb[1].p, 1, s));
            st = fine_bicgstab_l(h, 1, h->fb[1].p, z, s);
        }
        h->timer.stop(s);
        return st;
    }
    if (fp == 0) return vcycle0(h, 0, v, z, nb, s);
    CK(launch_convert_spinor(0, fp, g, v, h->fb[fp].p, nb, s));
    if (fp == 1) {
        TRY(vcycle0(h, 1, h->fb[1].p, z, nb, s));
        if (h->nn && !h->nn_off) {
            // learned correction of what the cycle leaves: z += N(v - D z)
            amg_dirac* d = h->d;
            CK(launch_dirac(1, g, nullptr, d->gauge->U[1].p, d->C[1].p, z, h->fx[1].p, h->fb[1].p, d->kappa, nb,
                            s));
            for (int q = 0; q < nb; ++q) {
                TRY(nn_forward_internal(h->nn, fld(h->fx[1], h, 1, q), h->nn->ework.p, s));
                CK(launch_axpby(1, make_double2(1, 0), h->nn->ework.p, make_double2(1, 0),
                                (char*)z + q * fsz(h, 1), fine_n(h), s));
            }
        }
        return AMG_OK;
    }
    TRY(vcycle0(h, fp, h->fb[fp].p, h->fx[fp].p, nb, s));
    CK(launch_convert_spinor(fp, 1, g, h->fx[fp].p, z, nb, s));
    return AMG_OK;
}

// w = D z for Z-precision z (FP64 result).  relaxed: the product may carry
// FP32 rounding (FP32 stencil, widened to FP64) -- see relaxed_product().
amg_status arnoldi_D(amg_hierarchy* h, const void* z, void* w, int nb, cudaStream_t s, bool relaxed = false) {
    if (zprec_of(h) == 0) return fine_D(h, 0, z, w, nullptr, nb, s);
    amg_dirac* d = h->d;
    if (relaxed) {
        CK(launch_dirac(1, fine_geom(h), nullptr, d->gauge->U[1].p, d->C[1].p, z, h->fx[1].p, nullptr, d->kappa, nb,
                        s));
        CK(launch_convert_spinor(1, 0, fine_geom(h), h->fx[1].p, w, nb, s));
        return AMG_OK;
    }
    CK(launch_dirac_mixed(fine_geom(h), d->gauge->U[3].p, d->C[3].p, z, w, d->kappa, nb, s));
    return AMG_OK;
}

// Relaxed Arnoldi products (inexact Krylov: the accuracy a product needs
// falls as the residual it has to reduce falls).  An error e_j in the j-th
// product moves the true residual away from the one the least-squares
// problem reports by at most |e_j| |y_j|, and |y_j| |D z_j| is about the
// residual r_j the step starts from.  With FP32 products (relative error
// ~6e-8, times the condition of D) the gap stays below 1e-3 tol |b| once
// |r_j| <= 1e-3 tol |b| / 6e-8; until then the product is FP64-accurate.  The
// FP64 true residual at the end of the cycle still decides convergence.
bool relaxed_product(double rel_residual, double tol) { return rel_residual <= 1e-3 * tol / 6e-8; }

// largest loss of orthogonality (eps |w| / |w'|) one classical Gram-Schmidt pass may leave
// before the outer solver projects a second time
constexpr double kReorthLoss = 1e-9;

// ---------------------------------------------------------------- outer FGMRES
// Flexible GMRES(m) in FP64 for nb right-hand sides in lockstep: one batched
// preconditioner call and one batched Arnoldi product per step, per-RHS
// Hessenberg / Givens / convergence; reductions of the whole batch share one
// host synchronisation.  A right-hand side that has converged (or stopped)
// rides along with a zero vector.
struct RhsState {
    double bnorm = 0, rn = 0, rel = 0;
    bool done = false, conv = false, stop = false;
    int iters = 0, restarts = 0, jend = -1;
    std::vector<std::vector<cplx>> H;
    std::vector<double> cs;
    std::vector<cplx> sn, g;
};

amg_status batch_norms(amg_hierarchy* h, int nb, const void* base, std::vector<double>& out, cudaStream_t s) {
    const size_t n = fine_n(h);
    Reducer& red = h->red;
    for (int q = 0; q < nb; ++q)
        CK(launch_norm2(0, (const char*)base + q * fsz(h, 0), n, (double*)red.dpart.p + (size_t)q * red.grid, s));
    CK(cudaMemcpyAsync(red.hpart, red.dpart.p, sizeof(double) * red.grid * nb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double* hp = (const double*)red.hpart;
    out.assign(nb, 0.0);
    for (int q = 0; q < nb; ++q)
        for (int i = 0; i < red.grid; ++i) out[q] += hp[(size_t)q * red.grid + i];
    return AMG_OK;
}

amg_status fgmres(amg_hierarchy* h, int nb, const void* b, void* x, bool x_nonzero, double tol, int maxit,
                  std::vector<amg_solve_info>& infos, cudaStream_t s) {
    const int m = h->p.outer_m;
    const size_t n = fine_n(h), fs = fsz(h, 0);
    Reducer& red = h->red;
    auto F = [&](const void* base, int q) { return (char*)base + q * fs; };
    std::vector<RhsState> st(nb);
    // ||b|| for every right-hand side
    {
        std::vector<double> bn2;
        TRY(batch_norms(h, nb, b, bn2, s));
        for (int q = 0; q < nb; ++q) {
            st[q].bnorm = std::sqrt(bn2[q]);
            if (st[q].bnorm == 0) {
                CK(cudaMemsetAsync(F(x, q), 0, fs, s));
                st[q].done = st[q].conv = true;
            }
        }
    }
    bool x_is_zero = !x_nonzero;
    while (true) {
        // true FP64 residual of every right-hand side
        std::vector<double> rn2(nb, 0.0);
        const void* rv = h->orr.p;   // the residual the cycle restarts from
        if (x_is_zero) {
            rv = b;   // r = b
            for (int q = 0; q < nb; ++q) rn2[q] = st[q].bnorm * st[q].bnorm;
            x_is_zero = false;
        } else {
            h->timer.start(PH_RESID, s);
            TRY(true_residual(h, x, h->orr.p, b, nb, s));   // r = b - D x
            h->timer.stop(s);
            TRY(batch_norms(h, nb, h->orr.p, rn2, s));
        }
        bool any = false;
        for (int q = 0; q < nb; ++q) {
            RhsState& r = st[q];
            if (r.bnorm == 0) continue;
            if (!std::isfinite(rn2[q])) return fail(AMG_NAN, "outer solve: non-finite residual");
            r.rn = std::sqrt(rn2[q]);
            r.rel = r.rn / r.bnorm;
            r.done = r.conv = r.rn <= tol * r.bnorm;
            if (!r.conv && r.iters >= maxit) r.done = true;
            if (!r.done) {
                any = true;
                if (r.iters > 0) r.restarts++;
            }
        }
        if (!any) break;
        // V_0 = r / |r| (zero for finished right-hand sides)
        for (int q = 0; q < nb; ++q) {
            RhsState& r = st[q];
            r.H.assign(m + 1, std::vector<cplx>(m, cplx(0)));
            r.cs.assign(m, 0.0);
            r.sn.assign(m, cplx(0));
            r.g.assign(m + 1, cplx(0));
            r.g[0] = r.rn;
            r.jend = -1;
            r.stop = r.done;
            if (r.done) CK(cudaMemsetAsync(F(h->oV[0]->p, q), 0, fs, s));
            else CK(launch_scale_real(0, 1.0 / r.rn, F(rv, q), F(h->oV[0]->p, q), n, s));
        }
        for (int j = 0; j < m; ++j) {
            TRY(precondition64(h, h->oV[j]->p, h->oZ[j]->p, nb, s));
            bool relax = true;
            for (int q = 0; q < nb; ++q)
                if (!st[q].stop) relax = relax && relaxed_product(std::abs(st[q].g[j]) / st[q].bnorm, tol);
            h->timer.start(PH_PROD, s);
            TRY(arnoldi_D(h, h->oZ[j]->p, h->ow.p, nb, s, relax));
            h->timer.stop(s);
            // classical Gram-Schmidt in FP64 with the coefficients summed on the device: the
            // dots, the update fused with |w'|^2, and the normalisation v_{j+1} = w' / |w'| run
            // back to back, and one host synchronisation per step fetches the Hessenberg
            // column.  One pass leaves v_{j+1} orthogonal to V up to about eps |w| / |w'|
            // (|w|^2 = |w'|^2 + sum |h_ij|^2); only if that exceeds kReorthLoss does a second
            // pass run (the Arnoldi relation D Z = V H holds to rounding either way, since every
            // update uses exactly the coefficients that enter H).
            std::vector<const void*> vl(j + 1);
            const size_t R = (size_t)20 * red.grid;
            double2* const gp = h->gs_part.as<double2>();
            double2* const gc = h->gs_coef.as<double2>();
            std::vector<double> hnv(nb, 0.0);   // |w'| exactly as the normalisation used it
            std::vector<char> again(nb, 0);
            // the last basis vector doubles as the copy-out staging of a host-vector solve's
            // previous batch: wait for that copy before overwriting it
            if (j + 1 == m && h->io_x_pending) CK(cudaStreamWaitEvent(s, h->io_ev[3], 0));
            for (int pass = 0; pass < 2; ++pass) {
                h->timer.start(PH_ORTH, s);
                bool any = false;
                for (int q = 0; q < nb; ++q) {
                    if (st[q].stop || (pass == 1 && !again[q])) continue;
                    any = true;
                    for (int i = 0; i <= j; ++i) vl[i] = F(h->oV[i]->p, q);
                    double2 *A = gp + (3 * q) * R, *C = gp + (3 * q + 2) * R;
                    double2* cu = gc + 64 * q + 32 * pass;
                    CK(launch_multi_dot(0, j + 1, vl.data(), F(h->ow.p, q), n, A, s));
                    CK(launch_multi_axpy_reduce_dev(0, j + 1, A, cu, vl.data(), F(h->ow.p, q), n, 0, C, s));
                    CK(launch_normalise(0, (const double*)C, (double*)(gc + 64 * q + 63), F(h->ow.p, q),
                                        F(h->oV[j + 1]->p, q), n, s));
                }
                h->timer.stop(s);
                if (!any) break;
                CK(cudaMemcpyAsync(h->gs_hcoef, gc, sizeof(double2) * 64 * nb, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                TRY(coarse_status(h));
                bool more = false;
                for (int q = 0; q < nb; ++q) {
                    RhsState& r = st[q];
                    if (r.stop || (pass == 1 && !again[q])) continue;
                    const double2* hc = h->gs_hcoef + 64 * q + 32 * pass;
                    double c2 = 0;
                    for (int i = 0; i <= j; ++i) {
                        r.H[i][j] += cplx(hc[i].x, hc[i].y);
                        c2 += hc[i].x * hc[i].x + hc[i].y * hc[i].y;
                    }
                    hnv[q] = reinterpret_cast<const double*>(h->gs_hcoef + 64 * q + 63)[0];
                    again[q] = pass == 0 && hnv[q] > 0 &&
                               2.2e-16 * std::sqrt(hnv[q] * hnv[q] + c2) > kReorthLoss * hnv[q];
                    more = more || again[q];
                }
                if (!more) break;
            }
            bool all_stopped = true;
            for (int q = 0; q < nb; ++q) {
                RhsState& r = st[q];
                if (r.stop) {
                    CK(cudaMemsetAsync(F(h->oV[j + 1]->p, q), 0, fs, s));
                    continue;
                }
                const double hn = hnv[q];
                auto& H = r.H;
                H[j + 1][j] = hn;
                r.iters++;
                for (int i = 0; i < j; ++i) {
                    cplx a = H[i][j], bb = H[i + 1][j];
                    H[i][j] = r.cs[i] * a + r.sn[i] * bb;
                    H[i + 1][j] = -std::conj(r.sn[i]) * a + r.cs[i] * bb;
                }
                {
                    cplx a = H[j][j], bb = H[j + 1][j];
                    double aa = std::abs(a), ab = std::abs(bb);
                    if (ab == 0) {
                        r.cs[j] = 1;
                        r.sn[j] = 0;
                    } else if (aa == 0) {
                        r.cs[j] = 0;
                        r.sn[j] = std::conj(bb) / ab;
                    } else {
                        double t = std::sqrt(aa * aa + ab * ab);
                        r.cs[j] = aa / t;
                        r.sn[j] = (a / aa) * std::conj(bb) / t;
                    }
                    H[j][j] = r.cs[j] * a + r.sn[j] * bb;
                    H[j + 1][j] = 0;
                    r.g[j + 1] = -std::conj(r.sn[j]) * r.g[j];
                    r.g[j] = r.cs[j] * r.g[j];
                }
                r.jend = j;
                const double est = std::abs(r.g[j + 1]);
                if (!std::isfinite(est)) return fail(AMG_NAN, "outer solve: non-finite Arnoldi coefficient");
                if (hn == 0 || est <= tol * r.bnorm || r.iters >= maxit) {
                    r.stop = true;
                    CK(cudaMemsetAsync(F(h->oV[j + 1]->p, q), 0, fs, s));
                } else {
                    all_stopped = false;   // v_{j+1} = w / |w| is already in place
                }
            }
            if (all_stopped) break;
        }
        // back substitution and x += Z y for every active right-hand side
        for (int q = 0; q < nb; ++q) {
            RhsState& r = st[q];
            if (r.done || r.jend < 0) continue;
            const int k = r.jend + 1;
            std::vector<cplx> y(k);
            for (int i = k - 1; i >= 0; --i) {
                cplx t = r.g[i];
                for (int c = i + 1; c < k; ++c) t -= r.H[i][c] * y[c];
                y[i] = t / r.H[i][i];
            }
            std::vector<double2> yc(k);
            std::vector<const void*> zl(k);
            for (int i = 0; i < k; ++i) {
                yc[i] = d2(y[i]);
                zl[i] = (const char*)h->oZ[i]->p + q * fsz(h, zprec_of(h));
            }
            if (zprec_of(h) == 0) CK(launch_multi_axpy(0, k, yc.data(), zl.data(), F(x, q), n, s));
            else CK(launch_spinor_axpy_mixed(fine_geom(h), k, yc.data(), zl.data(), F(x, q), s, true));
        }
    }
    infos.assign(nb, amg_solve_info());
    bool all_conv = true;
    for (int q = 0; q < nb; ++q) {
        std::memset(&infos[q], 0, sizeof(amg_solve_info));
        infos[q].iters = st[q].iters;
        infos[q].cycles = st[q].iters;
        infos[q].restarts = st[q].restarts;
        infos[q].converged = st[q].conv ? 1 : 0;
        infos[q].true_rel_residual = st[q].bnorm == 0 ? 0.0 : st[q].rel;
        all_conv = all_conv && st[q].conv;
    }
    return all_conv ? AMG_OK : AMG_NOT_CONVERGED;
}

// ---------------------------------------------------------------- setup pieces
// (Re)size the batch-dependent workspaces for nb right-hand sides.
// the coarse levels' solver fields for a batch of nb right-hand sides: [0] bc and [1] xc hold
// the batch, the coarsest solver's rt, R_j, U_j one lockstep group
constexpr int kSetupGroup = 4;   // test vectors per batched smoother / cycle call of the setup

amg_status alloc_coarse_workspaces(amg_hierarchy* h, int nb) {
    h->cw.resize(h->p.nlevels);
    for (int l = 1; l < h->p.nlevels; ++l) {
        CoarseLevel& L = h->lev[l];
        CK(L.cs_part.ensure(coarse_solver_partial_bytes()));
        if (!L.cs_state.p) {
            CK(L.cs_state.ensure(coarse_solver_state_bytes()));
            CK(cudaMemset(L.cs_state.p, 0, coarse_solver_state_bytes()));
        }
        size_t bytes = coarse_n(L) * coarse_elem_bytes(L.prec);
        int nv = 4 + 2 * (h->p.coarse_ell + 1);
        const int ng = l == h->p.nlevels - 1 ? std::min(nb, coarse_solver_max_rhs()) : 1;
        while ((int)h->cw[l].size() < nv) h->cw[l].push_back(new DevBuf());
        for (int k = 0; k < nv; ++k) CK(h->cw[l][k]->ensure(bytes * (k < 2 ? nb : ng)));
    }
    return AMG_OK;
}

amg_status alloc_workspaces(amg_hierarchy* h, int nb) {
    const GeomH& g = fine_geom(h);
    if (nb > h->nb_cap) h->clear_graphs();   // buffers may move: captured graphs would be stale
    TRY(h->red.init(nb));
    if (nb > h->gs_cap || !h->gs_hcoef) {
        CK(h->gs_part.ensure(sizeof(double2) * 3 * 20 * (size_t)blas_grid() * nb));
        CK(h->gs_coef.ensure(sizeof(double2) * 64 * nb));
        if (h->gs_hcoef) cudaFreeHost(h->gs_hcoef);
        h->gs_hcoef = nullptr;
        CK(cudaMallocHost(&h->gs_hcoef, sizeof(double2) * 64 * nb));
        h->gs_cap = nb;
    }
    CK(h->err_flag.ensure(sizeof(int)));
    // the batch runs its cycle in the smoother precision and its relaxed products in FP32; the
    // other precisions need one field each (conversions, the autotuner)
    for (int pr = 0; pr < 3; ++pr) {
        const int nf = (pr == h->fp || pr == 1) ? nb : 1;
        CK(h->fb[pr].ensure(fine_spinor_bytes(pr, g.V) * nf));
        CK(h->fx[pr].ensure(fine_spinor_bytes(pr, g.V) * nf));
    }
    CK(h->tmpv.ensure(fine_spinor_bytes(h->vp, g.V)));
    if (!h->hstate) {
        CK(cudaMallocHost(&h->hstate, 16 * 16));
        std::memset(h->hstate, 0, 16 * 16);
    }
    TRY(alloc_coarse_workspaces(h, nb));
    for (int l = 1; l + 1 < h->p.nlevels; ++l) {
        CoarseLevel& L = h->lev[l];
        const size_t bytes = coarse_n(L) * coarse_elem_bytes(L.prec);
        CK(L.cvecs.ensure(bytes * h->p.nvec[l]));
        L.gV.resize(h->p.inter_m + 1);
        L.gZ.resize(h->p.inter_m);
        for (auto& v : L.gV) CK(v.ensure(bytes));
        for (auto& z : L.gZ) CK(z.ensure(bytes));
        CK(L.gw.ensure(bytes));
        CK(L.gr.ensure(bytes));
        CK(L.gt.ensure(bytes));
    }
    const size_t fb64 = fine_spinor_bytes(0, g.V) * nb;
    CK(h->ob.ensure(fb64));
    CK(h->ox.ensure(fb64));
    CK(h->ow.ensure(fb64));
    CK(h->orr.ensure(fb64));
    while ((int)h->oV.size() < h->p.outer_m + 1) h->oV.push_back(new DevBuf());
    while ((int)h->oZ.size() < h->p.outer_m) h->oZ.push_back(new DevBuf());
    for (auto* v : h->oV) CK(v->ensure(fb64));
    for (auto* z : h->oZ) CK(z->ensure(fine_spinor_bytes(h->fp == 0 ? 0 : 1, g.V) * nb));
    if (h->p.outer_solver >= 1) {
        for (auto& v : h->bv) CK(v.ensure(fine_spinor_bytes(0, g.V)));
        for (auto& z : h->bz) CK(z.ensure(fine_spinor_bytes(h->fp == 0 ? 0 : 1, g.V)));
    }
    h->nb_cap = nb > h->nb_cap ? nb : h->nb_cap;
    return AMG_OK;
}

amg_status build_levels(amg_hierarchy* h) {
    const GeomH& g = fine_geom(h);
    h->lev.resize(h->p.nlevels);
    GeomH cur = g;
    for (int l = 0; l < h->p.nlevels - 1; ++l) {
        for (int mu = 0; mu < 4; ++mu) h->blk[l].b[mu] = h->p.block[l][mu];
        CoarseLevel& L = h->lev[l + 1];
        L.g.V = 1;
        for (int mu = 0; mu < 4; ++mu) {
            L.g.L[mu] = cur.L[mu] / h->p.block[l][mu];
            L.g.V *= L.g.L[mu];
        }
        L.g.antiperiodic = 0;
        L.nc = 2 * h->p.nvec[l];
        const bool last = l + 1 == h->p.nlevels - 1;
        L.opbf = last ? h->p.prec_coarsest == AMG_BF16 : h->p.prec_coarse == AMG_BF16;
        L.prec = last ? (h->p.prec_coarsest == AMG_F64 ? 0 : 1) : (h->p.prec_coarse == 0 ? 0 : 1);
        // the level whose vectors make this stencil: the fine level (test-vector precision) or level l
        const int producer = l == 0 ? h->vp : h->lev[l].prec;
        L.op32 = last && L.prec == 0 && producer == 1;
        const size_t ne = (size_t)L.g.V * 9 * L.nc * L.nc;
        CK(L.B.ensure(ne * coarse_elem_bytes(L.bprec())));
        if (L.opbf) CK(L.B16.ensure(ne * 4));
        cur = L.g;
    }
    CK(h->vecs0.ensure(fine_spinor_bytes(h->vp, g.V) * h->p.nvec[0]));
    return AMG_OK;
}

amg_status orthonormalise_and_galerkin(amg_hierarchy* h, cudaStream_t s) {
    const GeomH& g = fine_geom(h);
    CK(cudaMemsetAsync(h->err_flag.p, 0, sizeof(int), s));
    CK(launch_orthonormalise_fine(h->vp, g, h->blk[0], h->p.nvec[0], h->vecs0.p, h->err_flag.as<int>(), s));
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, h->err_flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (flag) return fail(AMG_EINVAL, "test vectors are rank deficient on some domain");
    if (h->rp == 2) {
        // round the orthonormalised vectors to half precision (per-site scale) and carry the
        // rounded values back, so that the Galerkin operator below, the restriction and the
        // prolongation all use the same vectors
        CK(h->vecs16.ensure(fine_spinor_bytes(2, g.V) * h->p.nvec[0]));
        CK(launch_convert_spinor(h->vp, 2, g, h->vecs0.p, h->vecs16.p, h->p.nvec[0], s));
        CK(launch_convert_spinor(2, h->vp, g, h->vecs16.p, h->vecs0.p, h->p.nvec[0], s));
    }
    amg_dirac* d = h->d;
    CoarseLevel& L = L1(h);
    CK(launch_galerkin_fine(h->vp, L.bprec(), g, h->blk[0], h->p.nvec[0], h->vecs0.p, d->gauge->U[h->vp].p,
                            d->C[h->vp].p, d->kappa, L.B.p, s));
    if (L.opbf) CK(launch_complex_to_bf16(L.B.p, L.B16.p, (size_t)L.g.V * 9 * L.nc * L.nc, s));
    if (L.opbf && coarse_tc_supported(L.nc)) {
        CK(L.tci.ensure(coarse_tc_image_bytes(L.g.V, L.nc)));
        CK(launch_coarse_tc_image(L.g.V, L.nc, L.B.p, L.tci.p, s));
    }
    return AMG_OK;
}

amg_status upload_vectors(amg_hierarchy* h, const double* host, cudaStream_t s) {
    const GeomH& g = fine_geom(h);
    const size_t cb = (size_t)g.V * 24 * sizeof(double);
    CK(h->canon.ensure(cb));
    const size_t vb = fine_spinor_bytes(h->vp, g.V);
    for (int i = 0; i < h->p.nvec[0]; ++i) {
        CK(cudaMemcpyAsync(h->canon.p, host + (size_t)i * g.V * 24, cb, cudaMemcpyDefault, s));
        if (h->vp == 0) {
            CK(launch_pack_spinor(0, g, h->canon.p, (char*)h->vecs0.p + i * vb, 1, s));
        } else {
            // canonical doubles -> P64 internal -> P32 internal
            CK(launch_pack_spinor(0, g, h->canon.p, h->fb[0].p, 1, s));
            CK(launch_convert_spinor(0, 1, g, h->fb[0].p, (char*)h->vecs0.p + i * vb, 1, s));
        }
    }
    CK(cudaStreamSynchronize(s));
    return AMG_OK;
}

amg_status normalise_into(amg_hierarchy* h, int prec, const void* src, void* dst, cudaStream_t s) {
    const size_t n = fine_n(h);
    double nn;
    TRY(h->red.norm2(prec, src, n, &nn, s));
    TRY(coarse_status(h));
    if (!(nn > 0) || !std::isfinite(nn)) return fail(AMG_NAN, "setup: test vector vanished or is not finite");
    CK(launch_axpby(prec, make_double2(1.0 / std::sqrt(nn), 0), src, make_double2(0, 0), dst, n, s));
    return AMG_OK;
}

// ---- setup of the levels between the fine and the coarsest grid
// level-l test vectors from host doubles [nvec][V_l][nc][re, im]
amg_status upload_cvecs(amg_hierarchy* h, int l, const double* host, cudaStream_t s) {
    CoarseLevel& L = h->lev[l];
    const size_t n = coarse_n(L) * h->p.nvec[l];
    if (L.prec == 0) {
        CK(cudaMemcpyAsync(L.cvecs.p, host, n * 16, cudaMemcpyDefault, s));
    } else {
        CK(h->canon.ensure(n * 16));
        CK(cudaMemcpyAsync(h->canon.p, host, n * 16, cudaMemcpyDefault, s));
        CK(launch_convert_flat(0, 1, h->canon.p, L.cvecs.p, n, s));
    }
    CK(cudaStreamSynchronize(s));
    return AMG_OK;
}

// Eq. 7 one level down: stencil of level l+1 from level l's stencil and vectors
amg_status galerkin_c(amg_hierarchy* h, int l, cudaStream_t s) {
    CoarseLevel& L = h->lev[l];
    CoarseLevel& N = h->lev[l + 1];
    CK(launch_galerkin_coarse(L.prec, N.bprec(), L.g, h->blk[l], L.nc, h->p.nvec[l], L.cvecs.p, L.B.p, N.B.p, s));
    if (N.opbf) CK(launch_complex_to_bf16(N.B.p, N.B16.p, (size_t)N.g.V * 9 * N.nc * N.nc, s));
    if (N.opbf && coarse_tc_supported(N.nc)) {
        CK(N.tci.ensure(coarse_tc_image_bytes(N.g.V, N.nc)));
        CK(launch_coarse_tc_image(N.g.V, N.nc, N.B.p, N.tci.p, s));
    }
    return AMG_OK;
}

amg_status ortho_galerkin_c(amg_hierarchy* h, int l, cudaStream_t s) {
    CoarseLevel& L = h->lev[l];
    CK(cudaMemsetAsync(h->err_flag.p, 0, sizeof(int), s));
    CK(launch_orthonormalise_coarse(L.prec, L.g, h->blk[l], L.nc, h->p.nvec[l], L.cvecs.p, h->err_flag.as<int>(),
                                    s));
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, h->err_flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (flag) return fail(AMG_EINVAL, "coarse test vectors are rank deficient on some domain");
    return galerkin_c(h, l, s);
}

// rebuild the stencils below level l after level l's stencil changed
amg_status refresh_c(amg_hierarchy* h, int l, cudaStream_t s) {
    for (int k = l; k + 1 < h->p.nlevels; ++k) TRY(galerkin_c(h, k, s));
    return AMG_OK;
}

amg_status normalise_c(amg_hierarchy* h, int l, const void* src, void* dst, cudaStream_t s) {
    CoarseLevel& L = h->lev[l];
    const size_t n = coarse_n(L);
    double nn;
    TRY(h->red.norm2(L.prec, src, n, &nn, s));
    TRY(coarse_status(h));
    if (!(nn > 0) || !std::isfinite(nn)) return fail(AMG_NAN, "setup: coarse test vector vanished or is not finite");
    CK(launch_axpby(L.prec, make_double2(1.0 / std::sqrt(nn), 0), src, make_double2(0, 0), dst, n, s));
    return AMG_OK;
}

// steps (0-a) and (0-b) on level l >= 1 (reading C6): smooth the level's
// initial vectors with its SAP, orthonormalise, build the next stencil, set up
// the next level, then n_adapt passes v <- M_l v with rebuilt stencils below
amg_status setup_coarse_level(amg_hierarchy* h, int l, const double* const* init, cudaStream_t s) {
    CoarseLevel& L = h->lev[l];
    if (!init[l]) return fail(AMG_EINVAL, "initial test vectors missing for a coarse level");
    TRY(upload_cvecs(h, l, init[l], s));
    const size_t vb = cvec_bytes(L);
    for (int k = 0; k < h->p.n_init; ++k)
        for (int i = 0; i < h->p.nvec[l]; ++i) {
            void* vi = (char*)L.cvecs.p + i * vb;
            TRY(coarse_sap(h, l, vi, L.gt.p, true, 1, s));
            TRY(normalise_c(h, l, L.gt.p, vi, s));
        }
    TRY(ortho_galerkin_c(h, l, s));
    if (l + 2 < h->p.nlevels) TRY(setup_coarse_level(h, l + 1, init, s));
    // every vector of a pass goes through the same cycle M_l (built from the vectors the pass
    // starts with): the new vectors are collected apart and replace the old ones at its end
    if (h->p.n_adapt > 0) CK(L.cvecs_next.ensure(vb * h->p.nvec[l]));
    for (int k = 0; k < h->p.n_adapt; ++k) {
        for (int i = 0; i < h->p.nvec[l]; ++i) {
            TRY(vcycle_c(h, l, (char*)L.cvecs.p + i * vb, L.gt.p, s));
            TRY(normalise_c(h, l, L.gt.p, (char*)L.cvecs_next.p + i * vb, s));
        }
        L.cvecs.swap(L.cvecs_next);
        TRY(ortho_galerkin_c(h, l, s));
        TRY(refresh_c(h, l + 1, s));
    }
    L.cvecs_next.release();
    return AMG_OK;
}

// Autotuner: for every smoother precision the hierarchy uses, time the SAP
// half-sweep variants on this lattice and blocking (zero fields; one full SAP
// iteration, both colours, per sample, the variants alternating so that drifts
// of clock or cache state hit both alike; the median of 9 samples decides),
// once for a single right-hand side and once for a batch of three (the staged
// variant shares its staged operator between two right-hand sides per CTA; an
// odd batch leaves half of its last CTAs idle, so three is its worst case), and
// keep the faster variant for each.
// Autotuner of the stencil's launch shape for precision pr (process-wide, dirac_set_shape):
// CTA size x grid cap from four candidates, then for FP32 / FP16 the 128-register budget for
// the best of them; median of two timed launches each on in -> out (fields of d's lattice)
amg_status tune_dirac_shape(amg_dirac* d, int pr, const void* in, void* out) {
    const GeomH& g = d->gauge->lat->g;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    std::vector<std::array<int, 3>> cand = {{256, 16, 0}, {128, 16, 0}, {256, 4, 0}, {128, 64, 0}};
    float best = 1e30f;
    int bt = 256, bs = 16, bm = 0;
    cudaError_t err = cudaSuccess;
    for (size_t ci = 0; ci < cand.size() && err == cudaSuccess; ++ci) {
        const auto c = cand[ci];
        dirac_set_shape(pr, c[0], c[1], c[2]);
        std::vector<float> t;
        for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
            err = cudaEventRecord(e0, 0);
            if (err == cudaSuccess)
                err = launch_dirac(pr, g, nullptr, d->gauge->U[pr].p, d->C[pr].p, in, out, nullptr, d->kappa, 1, 0);
            if (err == cudaSuccess) err = cudaEventRecord(e1, 0);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) t.push_back(ms);
        }
        if (err != cudaSuccess) break;
        std::sort(t.begin(), t.end());
        if (t[t.size() / 2] < best) {
            best = t[t.size() / 2];
            bt = c[0];
            bs = c[1];
            bm = c[2];
        }
        if (ci == 3 && pr != 0) cand.push_back({bt, bs, 2});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dirac_set_shape(pr, bt, bs, bm);
    CK(err);
    return AMG_OK;
}

amg_status tune_kernels(amg_hierarchy* h) {
    const GeomH& g = fine_geom(h);
    amg_dirac* d = h->d;
    int precs[2] = {h->fp, h->vp};
    for (int pr : precs) {
        const bool staged = sap_staged_supported(pr, h->blk[0]);
        if (h->p.sap_variant >= 0) {
            // variant 2 (two right-hand sides per CTA) only differs from 0 for batches; the
            // staged variants need a blocking that fits, 3 an FP32 smoother
            h->sap_variant[pr] = h->p.sap_variant == 2 ? 0 : h->p.sap_variant;
            h->sap_variant_nb[pr] = h->p.sap_variant;
            for (int* v : {&h->sap_variant[pr], &h->sap_variant_nb[pr]})
                if ((!staged && (*v == 1 || *v == 3)) || (*v == 3 && pr != 1)) *v = 0;
            continue;
        }
        const size_t fb = fine_spinor_bytes(pr, g.V);
        DevBuf tb, tx;
        CK(tb.ensure(3 * fb));
        CK(tx.ensure(3 * fb));
        CK(cudaMemset(tb.p, 0, 3 * fb));
        CK(cudaMemset(tx.p, 0, 3 * fb));
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        for (int nrhs : {1, 3}) {
            // candidates: 0 operator through L1/L2, 1 staged (if the blocking allows), and for
            // batches 2 (two right-hand sides per CTA through L1)
            std::vector<int> vs = {0};
            if (staged) vs.push_back(1);
            if (nrhs > 1) vs.push_back(2);
            if (staged && pr == 1) vs.push_back(3);
            std::vector<float> t[4];
            for (int rep = 0; rep < 10; ++rep) {
                for (int v : vs) {
                    CK(cudaEventRecord(e0, 0));
                    for (int colour = 0; colour < 2; ++colour)
                        CK(sap_half_launch(d, v, pr, g, h->blk[0], colour, h->p.mr_iters, 0, tb.p, tx.p, nrhs, 0));
                    CK(cudaEventRecord(e1, 0));
                    CK(cudaEventSynchronize(e1));
                    float ms = 0;
                    CK(cudaEventElapsedTime(&ms, e0, e1));
                    if (rep > 0) t[v].push_back(ms);
                }
            }
            int best_v = 0;
            float best_t = 1e30f;
            for (int v : vs) {
                std::sort(t[v].begin(), t[v].end());
                if (t[v][t[v].size() / 2] < best_t) {
                    best_t = t[v][t[v].size() / 2];
                    best_v = v;
                }
            }
            (nrhs == 1 ? h->sap_variant : h->sap_variant_nb)[pr] = best_v;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    // launch shape of the stencil (threads per CTA x grid cap x register budget) for the
    // precisions the solve applies D in: the smoother's (relaxed products) and FP64 (true residual)
    for (int pr : {h->fp, 0}) TRY(tune_dirac_shape(d, pr, h->fx[pr].p, h->fb[pr].p));
    return AMG_OK;
}

// Autotuner, second part (once the coarsest operator exists): the shared-memory tile of the
// coarsest solver -- coarse sites whose neighbour blocks are gathered per step -- timed over
// two BiCGStab(l) cycles (tolerance 0) on a fixed nonzero right-hand side per candidate.
amg_status tune_coarse_tile(amg_hierarchy* h) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // shared-memory tile of the coarsest solver: two BiCGStab(l) cycles (tolerance 0) on
    // a fixed nonzero right-hand side for each candidate
    const int lc = h->p.nlevels - 1;
    CoarseLevel& L = h->lev[lc];
    auto& w = h->cw[lc];
    const int ell = h->p.coarse_ell;
    void* R[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    void* Uv[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int j = 0; j <= ell; ++j) {
        R[j] = w[3 + j]->p;
        Uv[j] = w[4 + ell + j]->p;
    }
    CK(cudaMemset(w[0]->p, 0x3c, coarse_n(L) * coarse_elem_bytes(L.prec)));
    const int xmax = coarse_solver_max_xgroup(L.kprec(), L.nc, 1);
    std::vector<int> xs = {0};
    for (int xg : {xmax / 2, 4, 2, 1})
        if (xg >= 1 && xg < xmax && std::find(xs.begin(), xs.end(), xg) == xs.end()) xs.push_back(xg);
    float best = 1e30f;
    int bx = 0;
    for (int xg : xs) {
        std::vector<float> t;
        for (int rep = 0; rep < 3; ++rep) {
            CK(cudaMemset(L.cs_state.p, 0, 12));
            CK(cudaEventRecord(e0, 0));
            CK(launch_coarse_bicgstab(L.kprec(), L.g, L.nc, L.op(), w[0]->p, w[1]->p, w[2]->p, R, Uv, ell, 0.0, 2,
                                      L.cs_part.p, L.cs_state.p, 0, 0, 1, xg));
            CK(cudaEventRecord(e1, 0));
            CK(cudaEventSynchronize(e1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        if (t[t.size() / 2] < best) {
            best = t[t.size() / 2];
            bx = xg;
        }
    }
    L.xgroup = bx;
    CK(cudaMemset(L.cs_state.p, 0, 16));

    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return AMG_OK;
}

// A^{-1} of precision prec on the operator (FP64 inversion, once per precision)
amg_status ensure_clover_inverse(amg_dirac* d, int prec) {
    if (d->Ci[prec].p) return AMG_OK;
    const GeomH& g = d->gauge->lat->g;
    CK(d->Ci[prec].ensure(fine_clover_bytes(prec, g.V)));
    CK(launch_clover_invert(prec, g, d->C[0].p, d->Ci[prec].p, 0));
    CK(cudaStreamSynchronize(0));
    return AMG_OK;
}

amg_status hierarchy_init(amg_dirac* d, const amg_params* p, amg_hierarchy** out, amg_hierarchy** hp) {
    if (!d || !out) return fail(AMG_EINVAL, "NULL argument");
    TRY(check_params(d->gauge->lat->g, p));
    amg_hierarchy* h = new amg_hierarchy();
    h->d = d;
    h->p = *p;
    h->fp = p->prec_smoother;
    h->vp = vec_prec_of(p->prec_smoother);
    h->rp = p->prec_vectors == AMG_F16 ? 2 : h->vp;
    *hp = h;
    amg_status st = build_levels(h);
    if (st == AMG_OK && p->sap_eo) st = ensure_clover_inverse(d, h->fp);
    if (st == AMG_OK) st = alloc_workspaces(h, 1);
    if (st == AMG_OK) st = tune_kernels(h);
    if (st != AMG_OK) {
        delete h;
        *hp = nullptr;
        return st;
    }
    return AMG_OK;
}

// ---------------------------------------------------------------- flexible BiCGStab
// The paper's outer solver (Sec. 3): BiCGStab with the multigrid cycle as a
// flexible right preconditioner, two cycles and two Arnoldi-accurate products
// per iteration; the listing's misprints are read as in the standard method
// (x += omega M s, p = r + beta (p - omega D M p); reading C11).  The
// recursive residual ends an iteration sequence; the FP64 true residual
// b - D x then decides, and the method restarts from it if needed (C13).
// One right-hand side (field 0 of the outer workspaces).
amg_status fbicgstab(amg_hierarchy* h, const void* b, void* x, bool x_nonzero, double tol, int maxit,
                     amg_solve_info& info, cudaStream_t s) {
    const size_t n = fine_n(h), fs = fsz(h, 0);
    Reducer& red = h->red;
    void *r = h->bv[0].p, *rt = h->bv[1].p, *p = h->bv[2].p, *sv = h->bv[3].p, *t = h->bv[4].p, *dmp = h->bv[5].p;
    void *Mp = h->bz[0].p, *Ms = h->bz[1].p;
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
    auto add_z = [&](cplx c, const void* z) -> amg_status {   // x += c z
        double2 cc = d2(c);
        const void* zl[1] = {z};
        if (zprec_of(h) == 0) CK(launch_multi_axpy(0, 1, &cc, zl, x, n, s));
        else CK(launch_spinor_axpy_mixed(fine_geom(h), 1, &cc, zl, x, s));
        return AMG_OK;
    };
    std::memset(&info, 0, sizeof(info));
    double bn2;
    TRY(red.norm2(0, b, n, &bn2, s));
    if (!std::isfinite(bn2)) return fail(AMG_NAN, "outer solve: non-finite right-hand side");
    const double bn = std::sqrt(bn2);
    if (bn == 0) {
        CK(cudaMemsetAsync(x, 0, fs, s));
        info.converged = 1;
        return AMG_OK;
    }
    bool x_is_zero = !x_nonzero;
    int iters = 0;
    while (true) {
        double rn;
        if (x_is_zero) {
            CK(cudaMemcpyAsync(r, b, fs, cudaMemcpyDeviceToDevice, s));
            rn = bn;
            x_is_zero = false;
        } else {
            h->timer.start(PH_RESID, s);
            TRY(true_residual(h, x, r, b, 1, s));
            h->timer.stop(s);
            double rn2;
            TRY(red.norm2(0, r, n, &rn2, s));
            rn = std::sqrt(rn2);
        }
        if (!std::isfinite(rn)) return fail(AMG_NAN, "outer solve: non-finite residual");
        info.true_rel_residual = rn / bn;
        if (rn <= tol * bn) {
            info.converged = 1;
            break;
        }
        if (iters >= maxit) break;
        if (iters > 0) info.restarts++;
        CK(cudaMemcpyAsync(rt, r, fs, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(p, r, fs, cudaMemcpyDeviceToDevice, s));
        cplx rho = cplx(rn * rn, 0);
        while (iters < maxit) {
            TRY(precondition64(h, p, Mp, 1, s));
            ++info.cycles;
            h->timer.start(PH_PROD, s);
            TRY(arnoldi_D(h, Mp, dmp, 1, s));
            h->timer.stop(s);
            cplx den;
            TRY(red.dot(0, rt, dmp, n, &den, s));
            TRY(coarse_status(h));
            const cplx alpha = rho / den;
            if (!std::isfinite(alpha.real()) || !std::isfinite(alpha.imag()))
                return fail(AMG_NAN, "outer solve: BiCGStab breakdown");
            TRY(add_z(alpha, Mp));
            CK(cudaMemcpyAsync(sv, r, fs, cudaMemcpyDeviceToDevice, s));
            CK(launch_axpby(0, d2(-alpha), dmp, one, sv, n, s));
            ++iters;
            double sn2;
            TRY(red.norm2(0, sv, n, &sn2, s));
            if (std::sqrt(sn2) <= tol * bn) break;
            TRY(precondition64(h, sv, Ms, 1, s));
            ++info.cycles;
            h->timer.start(PH_PROD, s);
            TRY(arnoldi_D(h, Ms, t, 1, s));
            h->timer.stop(s);
            cplx ts;
            double tt;
            TRY(red.dot(0, t, sv, n, &ts, s));
            TRY(red.norm2(0, t, n, &tt, s));
            TRY(coarse_status(h));
            const cplx omega = ts / tt;
            if (!(tt > 0) || !std::isfinite(omega.real())) return fail(AMG_NAN, "outer solve: BiCGStab breakdown");
            TRY(add_z(omega, Ms));
            CK(cudaMemcpyAsync(r, sv, fs, cudaMemcpyDeviceToDevice, s));
            CK(launch_axpby(0, d2(-omega), t, one, r, n, s));
            // <r~, r> and |r|^2 in one pass
            const void* al[1] = {rt};
            CK(launch_multi_dot_norm(0, 1, al, r, n, red.dpart.as<double2>(), s));
            CK(cudaMemcpyAsync(red.hpart, red.dpart.p, sizeof(double2) * 2 * red.grid, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            cplx rho_new(0, 0);
            double rr = 0;
            for (int q = 0; q < red.grid; ++q) {
                rho_new += cplx(red.hpart[q].x, red.hpart[q].y);
                rr += red.hpart[red.grid + q].x;
            }
            if (std::sqrt(rr) <= tol * bn) break;
            const cplx beta = (alpha / omega) * (rho_new / rho);
            rho = rho_new;
            // p = r + beta (p - omega D M p)
            CK(launch_axpby(0, d2(-beta * omega), dmp, d2(beta), p, n, s));
            CK(launch_axpby(0, one, r, one, p, n, s));
            (void)zero;
        }
    }
    info.iters = iters;
    return info.converged ? AMG_OK : AMG_NOT_CONVERGED;
}

// the outer solver chosen by the parameters (flexible BiCGStab: nb == 1)
amg_status outer_solve(amg_hierarchy* h, int nb, const void* b, void* x, bool x_nonzero, double tol, int maxit,
                       std::vector<amg_solve_info>& infos, cudaStream_t s) {
    if (h->p.outer_solver == 0) return fgmres(h, nb, b, x, x_nonzero, tol, maxit, infos, s);
    if (nb != 1) return fail(AMG_EINVAL, "flexible BiCGStab solves one right-hand side at a time");
    // outer_solver 1: preconditioned by the multigrid cycle; 2 (MBiCGs): by BiCGStab(l) on D
    infos.assign(1, amg_solve_info());
    return fbicgstab(h, b, x, x_nonzero, tol, maxit, infos[0], s);
}

// ---------------------------------------------------------------- ragged batch
// Independent problems (each with its own lattice, operator and two-grid
// hierarchy) solved together: every phase of the outer flexible GMRES is
// issued for all active problems on a pool of streams before one host
// synchronisation.  Step j of a problem (Z_j = M V_j and w = D Z_j, about
// forty kernels) is replayed from a CUDA graph captured the first time; in it
// the coarse BiCGStab(l) runs as one thread-block cluster, so the problems'
// coarse solves overlap without a device-wide barrier.
amg_status ragged_step(amg_hierarchy* h, int j, cudaStream_t st) {
    if ((int)h->gexec.size() < h->p.outer_m) {
        h->gexec.resize(h->p.outer_m, nullptr);
        h->gkernels.resize(h->p.outer_m, 0);
    }
    if (!h->gexec[j]) {
        const unsigned long long k0 = g_launches.load(std::memory_order_relaxed);
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
        h->graph_mode = true;
        amg_status rc = precondition64(h, h->oV[j]->p, h->oZ[j]->p, 1, st);
        if (rc == AMG_OK) rc = arnoldi_D(h, h->oZ[j]->p, h->ow.p, 1, st);
        h->graph_mode = false;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc != AMG_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (rc != AMG_OK) return rc;
            CK(e);
        }
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        h->gexec[j] = ex;
        // kernels recorded during the capture ran no work: count them at every replay instead
        h->gkernels[j] = g_launches.load(std::memory_order_relaxed) - k0;
        g_launches.fetch_sub(h->gkernels[j], std::memory_order_relaxed);
    }
    CK(cudaGraphLaunch(h->gexec[j], st));
    g_launches.fetch_add(h->gkernels[j], std::memory_order_relaxed);
    return AMG_OK;
}

struct RaggedProb {
    amg_hierarchy* h = nullptr;
    cudaStream_t st = nullptr;
    RhsState r;
    bool started = false;   // true residual of x = 0 is b itself on the first cycle
    int coarse_cycles = 0;  // coarsest-level cycles (fused batches)
    // fused batches: the canonical vectors and the least-squares solution of the last cycle
    const double* bcanon = nullptr;
    double* xcanon = nullptr;
    std::vector<double2> y;
};

// partial sums of the last reduction launched for problem p (k values)
amg_status ragged_norm_launch(RaggedProb& p, const void* v) {
    Reducer& red = p.h->red;
    CK(launch_norm2(0, v, fine_n(p.h), (double*)red.dpart.p, p.st));
    CK(cudaMemcpyAsync(red.hpart, red.dpart.p, sizeof(double) * red.grid, cudaMemcpyDeviceToHost, p.st));
    return AMG_OK;
}
double ragged_norm_value(RaggedProb& p) {
    const double* hp = (const double*)p.h->red.hpart;
    double t = 0;
    for (int i = 0; i < p.h->red.grid; ++i) t += hp[i];
    return t;
}

amg_status fgmres_ragged(std::vector<RaggedProb>& P, const std::vector<cudaStream_t>& streams, double tol,
                         int maxit) {
    auto sync_all = [&]() -> amg_status {
        for (auto st : streams) CK(cudaStreamSynchronize(st));
        return AMG_OK;
    };
    int mmax = 0;
    for (auto& p : P) mmax = std::max(mmax, p.h->p.outer_m);
    // ||b||
    for (auto& p : P) TRY(ragged_norm_launch(p, p.h->ob.p));
    TRY(sync_all());
    for (auto& p : P) {
        p.r.bnorm = std::sqrt(ragged_norm_value(p));
        if (!std::isfinite(p.r.bnorm)) return fail(AMG_NAN, "ragged solve: non-finite right-hand side");
        if (p.r.bnorm == 0) p.r.done = p.r.conv = true;
    }
    while (true) {
        // true FP64 residual of every unfinished problem
        for (auto& p : P) {
            if (p.r.done) continue;
            if (p.started) {
                TRY(true_residual(p.h, p.h->ox.p, p.h->orr.p, p.h->ob.p, 1, p.st));
                TRY(ragged_norm_launch(p, p.h->orr.p));
            }
        }
        TRY(sync_all());
        bool any = false;
        for (auto& p : P) {
            RhsState& r = p.r;
            if (r.done) continue;
            TRY(coarse_status(p.h));
            const bool first = !p.started;   // x = 0: r = b
            r.rn = p.started ? std::sqrt(ragged_norm_value(p)) : r.bnorm;
            p.started = true;
            if (!std::isfinite(r.rn)) return fail(AMG_NAN, "ragged solve: non-finite residual");
            r.rel = r.rn / r.bnorm;
            r.done = r.conv = r.rn <= tol * r.bnorm;
            if (!r.conv && r.iters >= maxit) r.done = true;
            if (r.done) continue;
            any = true;
            if (r.iters > 0) r.restarts++;
            const int m = p.h->p.outer_m;
            r.H.assign(m + 1, std::vector<cplx>(m, cplx(0)));
            r.cs.assign(m, 0.0);
            r.sn.assign(m, cplx(0));
            r.g.assign(m + 1, cplx(0));
            r.g[0] = r.rn;
            r.jend = -1;
            r.stop = false;
            CK(launch_scale_real(0, 1.0 / r.rn, first ? p.h->ob.p : p.h->orr.p, p.h->oV[0]->p, fine_n(p.h),
                                 p.st));
        }
        if (!any) break;
        for (int j = 0; j < mmax; ++j) {
            bool active = false;
            for (auto& p : P) {
                if (p.r.done || p.r.stop) continue;
                if (j >= p.h->p.outer_m) {
                    p.r.stop = true;
                    continue;
                }
                active = true;
                TRY(ragged_step(p.h, j, p.st));
            }
            if (!active) break;
            // classical Gram-Schmidt in FP64 with device-side coefficients, as in fgmres: the
            // dots, the update fused with |w'|^2 and the normalisation per problem, one
            // synchronisation for the batch, and a second pass only where the loss of
            // orthogonality estimate asks for it (reading C23)
            const size_t R = (size_t)20 * blas_grid();
            std::vector<char> in(P.size(), 0), again(P.size(), 0);
            std::vector<double> hnv(P.size(), 0.0);
            for (size_t t = 0; t < P.size(); ++t) in[t] = !(P[t].r.done || P[t].r.stop);
            for (int pass = 0; pass < 2; ++pass) {
                bool any_pass = false;
                for (size_t t = 0; t < P.size(); ++t) {
                    RaggedProb& p = P[t];
                    if (!in[t] || (pass == 1 && !again[t])) continue;
                    any_pass = true;
                    std::vector<const void*> vl(j + 1);
                    for (int i = 0; i <= j; ++i) vl[i] = p.h->oV[i]->p;
                    double2* gp = p.h->gs_part.as<double2>();
                    double2* gc = p.h->gs_coef.as<double2>();
                    const size_t n = fine_n(p.h);
                    CK(launch_multi_dot(0, j + 1, vl.data(), p.h->ow.p, n, gp, p.st));
                    CK(launch_multi_axpy_reduce_dev(0, j + 1, gp, gc + 32 * pass, vl.data(), p.h->ow.p, n, 0,
                                                    gp + 2 * R, p.st));
                    CK(launch_normalise(0, (const double*)(gp + 2 * R), (double*)(gc + 63), p.h->ow.p,
                                        p.h->oV[j + 1]->p, n, p.st));
                    CK(cudaMemcpyAsync(p.h->gs_hcoef, gc, sizeof(double2) * 64, cudaMemcpyDeviceToHost, p.st));
                }
                if (!any_pass) break;
                TRY(sync_all());
                bool more = false;
                for (size_t t = 0; t < P.size(); ++t) {
                    RaggedProb& p = P[t];
                    if (!in[t] || (pass == 1 && !again[t])) continue;
                    if (pass == 0) TRY(coarse_status(p.h));
                    const double2* hc = p.h->gs_hcoef + 32 * pass;
                    double c2 = 0;
                    for (int i = 0; i <= j; ++i) {
                        p.r.H[i][j] += cplx(hc[i].x, hc[i].y);
                        c2 += hc[i].x * hc[i].x + hc[i].y * hc[i].y;
                    }
                    hnv[t] = reinterpret_cast<const double*>(p.h->gs_hcoef + 63)[0];
                    again[t] = pass == 0 && hnv[t] > 0 &&
                               2.2e-16 * std::sqrt(hnv[t] * hnv[t] + c2) > kReorthLoss * hnv[t];
                    more = more || again[t];
                }
                if (!more) break;
            }
            for (size_t t = 0; t < P.size(); ++t) {
                RaggedProb& p = P[t];
                RhsState& r = p.r;
                if (r.done || r.stop) continue;
                const double hn = hnv[t];
                r.H[j + 1][j] = hn;
                r.iters++;
                givens_column(r.H, r.cs, r.sn, r.g, j);
                r.jend = j;
                const double est = std::abs(r.g[j + 1]);
                if (!std::isfinite(est)) return fail(AMG_NAN, "ragged solve: non-finite Arnoldi coefficient");
                if (hn == 0 || est <= tol * r.bnorm || r.iters >= maxit) r.stop = true;   // else v_{j+1} is in place
            }
        }
        // x += Z y
        for (auto& p : P) {
            RhsState& r = p.r;
            if (r.done || r.jend < 0) continue;
            const int k = r.jend + 1;
            std::vector<cplx> y(k);
            for (int i = k - 1; i >= 0; --i) {
                cplx t = r.g[i];
                for (int cc = i + 1; cc < k; ++cc) t -= r.H[i][cc] * y[cc];
                y[i] = t / r.H[i][i];
            }
            std::vector<double2> yc(k);
            std::vector<const void*> zl(k);
            for (int i = 0; i < k; ++i) {
                yc[i] = d2(y[i]);
                zl[i] = p.h->oZ[i]->p;
            }
            if (zprec_of(p.h) == 0) CK(launch_multi_axpy(0, k, yc.data(), zl.data(), p.h->ox.p, fine_n(p.h), p.st));
            else CK(launch_spinor_axpy_mixed(fine_geom(p.h), k, yc.data(), zl.data(), p.h->ox.p, p.st));
        }
    }
    return AMG_OK;
}


// ---------------------------------------------------------------- fused ragged batch
// The same lockstep flexible GMRES with every phase of an Arnoldi step issued
// as ONE launch for all active problems: a table of per-problem descriptors
// (ragged_dev_fill) and per-phase prefix tables of CTA offsets split each grid
// among the problems, so a problem of 4^4 sites and one of 16^3 x 32 share a
// launch.  Per step: FP64 -> FP32 copy of V_j, restriction, the coarse
// BiCGStab(l) (one thread-block cluster per problem in one launch), prolongation,
// 2 sap_iters SAP half sweeps, the FP64-accurate Arnoldi product and a
// classical Gram-Schmidt pass -- 2 sap_iters + 8 kernels for the whole batch,
// whatever its size.  Used when every problem has an FP32 smoother, FP32
// coarse vectors, the same coarse operator storage and test-vector precision,
// blocks of at most 256 sites and outer_m < 20 (else the stream pool above).
bool g_ragged_fused = true;   // amg_set_ragged_fusion

struct FusedBatch {
    enum { T_SITE, T_BLK, T_DOM, T_BLAS, NT };
    static constexpr int kSlots = 4;   // host staging slots, reused in turn once their copy is done
    size_t db = 0, sb = 0, slot_bytes = 0;
    int cap = 0, next = 0;
    DevBuf desc, off, cargs, cstate, coef;
    char* hstage = nullptr;      // pinned: kSlots x (descriptors, offset tables)
    cudaEvent_t ev[kSlots] = {};
    char* hstate = nullptr;      // pinned: coarse solver state words, Gram-Schmidt coefficients,
    double2* hcoef = nullptr;    // coarse solver arguments (rewritten once per step, after a sync)
    void* hcargs = nullptr;
    int max_vb = 0, max_nvec = 0;
    ~FusedBatch() {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
        if (hstage) cudaFreeHost(hstage);
        if (hstate) cudaFreeHost(hstate);
        if (hcoef) cudaFreeHost(hcoef);
        if (hcargs) cudaFreeHost(hcargs);
    }
    // two device regions of cap problems each: the step's active set (0), and the sets of the
    // restart phases and of a second Gram-Schmidt pass (1)
    amg_status alloc(int n) {
        db = ragged_dev_bytes();
        sb = coarse_solver_state_bytes();
        cap = n;
        slot_bytes = (db * n + sizeof(int) * NT * (n + 1) + 255) / 256 * 256;
        CK(desc.ensure(2 * db * n));
        CK(off.ensure(sizeof(int) * 2 * NT * (n + 1)));
        CK(cargs.ensure(coarse_solver_desc_bytes() * n));
        CK(cstate.ensure(sb * n));
        CK(coef.ensure(sizeof(double2) * 64 * n));
        CK(cudaMallocHost((void**)&hstage, slot_bytes * kSlots));
        for (auto& e : ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        CK(cudaMallocHost((void**)&hstate, sb * n));
        CK(cudaMallocHost((void**)&hcoef, sizeof(double2) * 64 * n));
        CK(cudaMallocHost(&hcargs, coarse_solver_desc_bytes() * n));
        return AMG_OK;
    }
    const void* d(int region) const { return (const char*)desc.p + region * db * cap; }
    const int* o(int region, int t) const { return off.as<int>() + (region * NT + t) * (cap + 1); }
};

bool fusable(const std::vector<RaggedProb>& P) {
    const amg_hierarchy* h0 = P[0].h;
    for (const auto& p : P) {
        const amg_hierarchy* h = p.h;
        const CoarseLevel& L = h->lev[1];
        int vb = 1;
        for (int mu = 0; mu < 4; ++mu) vb *= h->blk[0].b[mu];
        if (h->fp != 1 || h->p.sap_eo || L.prec != 1 || L.kprec() != h0->lev[1].kprec() || h->rp != h0->rp ||
            vb > 256 || h->p.outer_m + 1 > 20 || h->p.coarse_ell > 4 || h->nn)
            return false;
        if (h->p.sap_iters != h0->p.sap_iters || h->p.mr_iters != h0->p.mr_iters) return false;
        if (h->p.resid_pair != h0->p.resid_pair) return false;
        if (!h->d->gauge->U[3].p || !h->d->C[3].p || !h->d->gauge->U[1].p || !h->d->C[1].p) return false;
    }
    return true;
}

// descriptors and CTA offset tables of the problems idx at Arnoldi step j into region r
// (uploaded on st); the Gram-Schmidt coefficients of problem i live at coef + 64 i
amg_status fused_tables(FusedBatch& F, std::vector<RaggedProb>& P, const std::vector<int>& idx, int j, int r,
                        int tot[FusedBatch::NT], cudaStream_t st) {
    const int na = (int)idx.size(), stride = F.cap + 1;
    // a staging slot whose last upload has been done
    const int slot = F.next;
    F.next = (F.next + 1) % FusedBatch::kSlots;
    CK(cudaEventSynchronize(F.ev[slot]));
    char* hd = F.hstage + slot * F.slot_bytes;
    int* ho = reinterpret_cast<int*>(hd + F.db * F.cap);
    for (int t = 0; t < FusedBatch::NT; ++t) tot[t] = 0;
    for (int a = 0; a < na; ++a) {
        amg_hierarchy* h = P[idx[a]].h;
        amg_dirac* d = h->d;
        const GeomH& g = fine_geom(h);
        CoarseLevel& L = h->lev[1];
        RaggedProbH q = {};
        q.g = g;
        q.blk = h->blk[0];
        q.nvec = h->p.nvec[0];
        q.kappa = d->kappa;
        q.U32 = d->gauge->U[1].p;
        q.C32 = d->C[1].p;
        q.Udd = d->gauge->U[3].p;
        q.Cdd = d->C[3].p;
        q.vecs = rp_vecs(h);
        q.v = h->oV[j]->p;
        q.f32 = h->fb[1].p;
        q.f32b = h->fx[1].p;
        q.bc = h->cw[1][0]->p;
        q.xc = h->cw[1][1]->p;
        q.z = h->oZ[j]->p;
        q.w = h->ow.p;
        for (int i = 0; i <= j; ++i) q.basis[i] = h->oV[i]->p;
        q.nbasis = j + 1;
        q.vnext = h->oV[j + 1]->p;
        q.gs_part = h->gs_part.as<double2>();
        q.gs_coef = F.coef.as<double2>() + 64 * (size_t)idx[a];
        q.n = fine_n(h);
        q.R = (size_t)20 * blas_grid();
        q.U64 = d->gauge->U[0].p;
        q.C64 = d->C[0].p;
        q.b64 = h->ob.p;
        q.x64 = h->ox.p;
        q.r64 = h->orr.p;
        q.rsrc = P[idx[a]].started ? h->orr.p : h->ob.p;
        q.npart = reinterpret_cast<double*>(h->gs_part.as<double2>() + 2 * q.R);
        q.nval = reinterpret_cast<double*>(F.coef.as<double2>() + 64 * (size_t)idx[a] + 62);
        q.k = (int)P[idx[a]].y.size();
        for (int i = 0; i < q.k; ++i) {
            q.zb[i] = h->oZ[i]->p;
            q.yc[i] = P[idx[a]].y[i];
        }
        q.canon_in = P[idx[a]].bcanon;
        q.canon_out = P[idx[a]].xcanon;
        int vb = 1;
        for (int mu = 0; mu < 4; ++mu) vb *= h->blk[0].b[mu];
        q.sap_nr = ragged_sap_nr(vb, F.max_vb);
        if (ragged_dev_fill(hd + (size_t)a * F.db, q) != 0)
            return fail(AMG_EINVAL, "ragged solve: bad problem descriptor");
        const int nt[FusedBatch::NT] = {ragged_site_ctas(g.V), L.g.V, (L.g.V / 2 + q.sap_nr - 1) / q.sap_nr,
                                        ragged_blas_ctas(q.n)};
        for (int t = 0; t < FusedBatch::NT; ++t) {
            ho[t * stride + a] = tot[t];
            tot[t] += nt[t];
        }
    }
    for (int t = 0; t < FusedBatch::NT; ++t) ho[t * stride + na] = tot[t];
    CK(cudaMemcpyAsync((char*)F.desc.p + (size_t)r * F.cap * F.db, hd, na * F.db, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(F.off.as<int>() + r * FusedBatch::NT * stride, ho, sizeof(int) * FusedBatch::NT * stride,
                       cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(F.ev[slot], st));
    return AMG_OK;
}

// Z_j = M V_j and w = D Z_j for the problems of region 0 (na of them, step tables tot)
amg_status fused_precondition(FusedBatch& F, std::vector<RaggedProb>& P, const std::vector<int>& act,
                              const int tot[FusedBatch::NT], cudaStream_t st) {
    const int na = (int)act.size();
    const void* d = F.d(0);
    amg_hierarchy* h0 = P[act[0]].h;
    CK(launch_convert_ragged(d, F.o(0, FusedBatch::T_SITE), na, tot[FusedBatch::T_SITE], st));
    CK(launch_restrict_ragged(h0->rp, d, F.o(0, FusedBatch::T_BLK), na, tot[FusedBatch::T_BLK], F.max_vb, F.max_nvec,
                              st));
    std::vector<CoarseSolveDesc> cd(na);
    for (int a = 0; a < na; ++a) {
        amg_hierarchy* h = P[act[a]].h;
        CoarseLevel& L = h->lev[1];
        auto& w = h->cw[1];
        const int ell = h->p.coarse_ell;
        CoarseSolveDesc& c = cd[a];
        c.cprec = L.kprec();
        c.gc = L.g;
        c.nc = L.nc;
        c.B = L.op();
        c.b = w[0]->p;
        c.x = w[1]->p;
        c.rt = w[2]->p;
        for (int k = 0; k < 5; ++k) {
            c.R[k] = k <= ell ? w[3 + k]->p : nullptr;
            c.U[k] = k <= ell ? w[4 + ell + k]->p : nullptr;
        }
        c.ell = ell;
        c.tol = h->p.coarse_tol;
        c.maxit = h->p.coarse_maxit;
        c.part = L.cs_part.p;
        c.state = (char*)F.cstate.p + a * F.sb;
        c.xgroup = L.xgroup;
    }
    CK(cudaMemsetAsync(F.cstate.p, 0, F.sb * na, st));
    CK(launch_coarse_bicgstab_multi(cd.data(), na, F.hcargs, F.cargs.p, st));
    CK(cudaMemcpyAsync(F.hstate, F.cstate.p, F.sb * na, cudaMemcpyDeviceToHost, st));
    CK(launch_prolong_ragged(h0->rp, d, F.o(0, FusedBatch::T_BLK), na, tot[FusedBatch::T_BLK], F.max_vb, F.max_nvec,
                             st));
    for (int i = 0; i < h0->p.sap_iters; ++i)
        for (int colour = 0; colour < 2; ++colour)
            CK(launch_sap_half_ragged(d, F.o(0, FusedBatch::T_DOM), na, tot[FusedBatch::T_DOM], F.max_vb, colour,
                                      h0->p.mr_iters, st));
    CK(launch_dirac_mixed_ragged(d, F.o(0, FusedBatch::T_SITE), na, tot[FusedBatch::T_SITE], st));
    return AMG_OK;
}

amg_status fgmres_fused(std::vector<RaggedProb>& P, cudaStream_t st, double tol, int maxit) {
    const int n = (int)P.size();
    FusedBatch F;
    TRY(F.alloc(n));
    int mmax = 0;
    for (auto& p : P) {
        p.st = st;
        mmax = std::max(mmax, p.h->p.outer_m);
        int vb = 1;
        for (int mu = 0; mu < 4; ++mu) vb *= p.h->blk[0].b[mu];
        F.max_vb = std::max(F.max_vb, vb);
        F.max_nvec = std::max(F.max_nvec, p.h->p.nvec[0]);
    }
    int tot0[FusedBatch::NT], tot1[FusedBatch::NT];
    std::vector<int> all(n);
    for (int i = 0; i < n; ++i) all[i] = i;
    // b and x = 0 in the internal layout
    TRY(fused_tables(F, P, all, 0, 1, tot1, st));
    CK(launch_pack_ragged(F.d(1), F.o(1, FusedBatch::T_SITE), n, tot1[FusedBatch::T_SITE], st));
    bool first = true;
    while (true) {
        // true FP64 residual of every unfinished problem (b itself while x = 0), its norm and
        // V_0 = r / |r|: three launches for the set, one synchronisation
        std::vector<int> set;
        for (int i = 0; i < n; ++i)
            if (!P[i].r.done) set.push_back(i);
        if (set.empty()) break;
        TRY(fused_tables(F, P, set, 0, 1, tot1, st));
        const int ns = (int)set.size();
        if (!first)
            CK(launch_resid_ragged(F.d(1), F.o(1, FusedBatch::T_SITE), ns, tot1[FusedBatch::T_SITE],
                                   P[0].h->p.resid_pair != 0, st));
        CK(launch_norm_v0_ragged(F.d(1), F.o(1, FusedBatch::T_BLAS), ns, tot1[FusedBatch::T_BLAS], st));
        CK(cudaMemcpyAsync(F.hcoef, F.coef.p, sizeof(double2) * 64 * n, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        bool any = false;
        for (int i : set) {
            RaggedProb& p = P[i];
            RhsState& r = p.r;
            const double nv = reinterpret_cast<const double*>(F.hcoef + 64 * i + 62)[0];
            if (first) {
                r.bnorm = nv;
                if (!std::isfinite(r.bnorm)) return fail(AMG_NAN, "ragged solve: non-finite right-hand side");
                if (r.bnorm == 0) {
                    r.done = r.conv = true;
                    continue;
                }
            }
            p.started = true;
            r.rn = nv;
            if (!std::isfinite(r.rn)) return fail(AMG_NAN, "ragged solve: non-finite residual");
            r.rel = r.rn / r.bnorm;
            r.done = r.conv = r.rn <= tol * r.bnorm;
            if (!r.conv && r.iters >= maxit) r.done = true;
            if (r.done) continue;
            any = true;
            if (r.iters > 0) r.restarts++;
            const int m = p.h->p.outer_m;
            r.H.assign(m + 1, std::vector<cplx>(m, cplx(0)));
            r.cs.assign(m, 0.0);
            r.sn.assign(m, cplx(0));
            r.g.assign(m + 1, cplx(0));
            r.g[0] = r.rn;
            r.jend = -1;
            r.stop = false;
        }
        first = false;
        if (!any) break;
        for (int j = 0; j < mmax; ++j) {
            std::vector<int> act;
            for (int i = 0; i < n; ++i) {
                RaggedProb& p = P[i];
                if (p.r.done || p.r.stop) continue;
                if (j >= p.h->p.outer_m) {
                    p.r.stop = true;
                    continue;
                }
                act.push_back(i);
            }
            if (act.empty()) break;
            const int na = (int)act.size();
            TRY(fused_tables(F, P, act, j, 0, tot0, st));
            TRY(fused_precondition(F, P, act, tot0, st));
            // classical Gram-Schmidt in FP64 (reading C23), one launch per kernel for the batch;
            // a second pass only for the problems whose loss-of-orthogonality estimate asks for it
            CK(launch_gs_ragged(j + 1, F.d(0), F.o(0, FusedBatch::T_BLAS), na, tot0[FusedBatch::T_BLAS], 0, st));
            CK(cudaMemcpyAsync(F.hcoef, F.coef.p, sizeof(double2) * 64 * n, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            for (int a = 0; a < na; ++a) {
                const int* w = reinterpret_cast<const int*>(F.hstate + a * F.sb);
                if (w[2] == 1) return fail(AMG_TIMEOUT, "coarse solver: grid barrier timed out");
                if (w[2] != 0) return fail(AMG_NAN, "coarse solver: breakdown or non-finite residual");
                P[act[a]].coarse_cycles += w[3];
            }
            std::vector<int> again;
            std::vector<double> hnv(n, 0.0);
            for (int pass = 0; pass < 2; ++pass) {
                const std::vector<int>& set = pass == 0 ? act : again;
                std::vector<int> more;
                for (int i : set) {
                    RaggedProb& p = P[i];
                    const double2* hc = F.hcoef + 64 * i + 32 * pass;
                    double c2 = 0;
                    for (int k = 0; k <= j; ++k) {
                        p.r.H[k][j] += cplx(hc[k].x, hc[k].y);
                        c2 += hc[k].x * hc[k].x + hc[k].y * hc[k].y;
                    }
                    hnv[i] = reinterpret_cast<const double*>(F.hcoef + 64 * i + 63)[0];
                    if (pass == 0 && hnv[i] > 0 && 2.2e-16 * std::sqrt(hnv[i] * hnv[i] + c2) > kReorthLoss * hnv[i])
                        more.push_back(i);
                }
                if (pass == 1 || more.empty()) break;
                again = more;
                TRY(fused_tables(F, P, again, j, 1, tot1, st));
                CK(launch_gs_ragged(j + 1, F.d(1), F.o(1, FusedBatch::T_BLAS), (int)again.size(),
                                    tot1[FusedBatch::T_BLAS], 1, st));
                CK(cudaMemcpyAsync(F.hcoef, F.coef.p, sizeof(double2) * 64 * n, cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
            }
            for (int i : act) {
                RhsState& r = P[i].r;
                const double hn = hnv[i];
                r.H[j + 1][j] = hn;
                r.iters++;
                givens_column(r.H, r.cs, r.sn, r.g, j);
                r.jend = j;
                const double est = std::abs(r.g[j + 1]);
                if (!std::isfinite(est)) return fail(AMG_NAN, "ragged solve: non-finite Arnoldi coefficient");
                if (hn == 0 || est <= tol * r.bnorm || r.iters >= maxit) r.stop = true;
            }
        }
        // x += Z y: one launch for every problem that took steps in this cycle
        std::vector<int> upd;
        for (int i = 0; i < n; ++i) {
            RaggedProb& p = P[i];
            RhsState& r = p.r;
            p.y.clear();
            if (r.done || r.jend < 0) continue;
            const int k = r.jend + 1;
            std::vector<cplx> y(k);
            for (int a = k - 1; a >= 0; --a) {
                cplx t = r.g[a];
                for (int cc = a + 1; cc < k; ++cc) t -= r.H[a][cc] * y[cc];
                y[a] = t / r.H[a][a];
            }
            p.y.resize(k);
            for (int a = 0; a < k; ++a) p.y[a] = d2(y[a]);
            upd.push_back(i);
        }
        if (!upd.empty()) {
            TRY(fused_tables(F, P, upd, 0, 1, tot1, st));
            CK(launch_xupdate_ragged(F.d(1), F.o(1, FusedBatch::T_SITE), (int)upd.size(), tot1[FusedBatch::T_SITE],
                                     st));
        }
    }
    TRY(fused_tables(F, P, all, 0, 1, tot1, st));
    CK(launch_unpack_ragged(F.d(1), F.o(1, FusedBatch::T_SITE), n, tot1[FusedBatch::T_SITE], st));
    return AMG_OK;
}
}  // namespace

// accessors used by the allocation-free entry point (noalloc.cu)
const GeomH* amg_internal_geom(const amg_dirac* d) { return &d->gauge->lat->g; }
const void* amg_internal_links(const amg_dirac* d, int prec) { return d->gauge->U[prec].p; }
const void* amg_internal_clover(const amg_dirac* d, int prec) { return d->C[prec].p; }
double amg_internal_kappa(const amg_dirac* d) { return d->kappa; }
amg_dirac* amg_internal_hierarchy_dirac(amg_hierarchy* h) { return h->d; }
void amg_internal_set_error(const char* msg) { g_err = msg; }

// ================================================================ C ABI

extern "C" {

const char* amg_last_error(void) { return g_err.c_str(); }

unsigned long long amg_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

void amg_params_default(amg_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nlevels = 2;
    for (int l = 0; l < AMG_MAX_LEVELS - 1; ++l) {
        for (int mu = 0; mu < 4; ++mu) p->block[l][mu] = 4;
        p->nvec[l] = 24;
    }
    p->n_init = 3;
    p->n_adapt = 2;
    p->sap_iters = 4;
    p->mr_iters = 6;
    p->coarse_tol = 1e-2;
    p->coarse_maxit = 200;
    p->coarse_ell = 2;
    p->inter_m = 8;
    p->inter_tol = 1e-1;
    p->inter_maxit = 8;
    p->outer_m = 16;
    p->prec_smoother = AMG_F32;
    p->prec_coarse = AMG_F32;
    p->prec_coarsest = AMG_F32;
    p->sap_variant = -1;
    p->outer_solver = 0;
    p->prec_vectors = AMG_F32;
    p->mbicgs_tol = 1e-4;
    p->mbicgs_maxit = 50;
    p->sap_eo = 0;
    p->coarse_tc = 0;
    p->resid_pair = 0;
}


amg_status amg_lattice_create(const int dims[4], int antiperiodic_t, amg_lattice** out) {
    if (!dims || !out) return fail(AMG_EINVAL, "NULL argument");
    long long V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2) return fail(AMG_EINVAL, "lattice extents must be >= 2");
        V *= dims[mu];
    }
    if (V > (1ll << 30)) return fail(AMG_EINVAL, "lattice too large");
    amg_lattice* l = new amg_lattice();
    for (int mu = 0; mu < 4; ++mu) l->g.L[mu] = dims[mu];
    l->g.V = (int)V;
    l->g.antiperiodic = antiperiodic_t ? 1 : 0;
    *out = l;
    return AMG_OK;
}
void amg_lattice_destroy(amg_lattice* l) { delete l; }

// gauge handle from canonical double links already on the device
static amg_status gauge_from_device(amg_lattice* lat, const double* canon, amg_gauge** out) {
    const GeomH& g = lat->g;
    amg_gauge* G = new amg_gauge();
    G->lat = lat;
    for (int pr = 0; pr < 4; ++pr) {
        if (G->U[pr].ensure(fine_gauge_bytes(pr, g.V)) != cudaSuccess) {
            delete G;
            return fail(AMG_ENOMEM, "gauge: device allocation failed");
        }
        if (launch_gauge_convert(pr, g, canon, G->U[pr].p, 0) != cudaSuccess) {
            delete G;
            return fail(AMG_ECUDA, "gauge: conversion kernel failed");
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        delete G;
        return fail(AMG_ECUDA, "gauge: conversion failed");
    }
    *out = G;
    return AMG_OK;
}

amg_status amg_gauge_create(amg_lattice* lat, const double* U_host, amg_gauge** out) {
    if (!lat || !U_host || !out) return fail(AMG_EINVAL, "NULL argument");
    const GeomH& g = lat->g;
    DevBuf canon;
    size_t cb = (size_t)g.V * 4 * 18 * sizeof(double);
    if (canon.ensure(cb) != cudaSuccess) return fail(AMG_ENOMEM, "gauge: device allocation failed");
    if (cudaMemcpy(canon.p, U_host, cb, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(AMG_ECUDA, "gauge: upload failed");
    return gauge_from_device(lat, canon.as<double>(), out);
}

amg_status amg_gauge_random(amg_lattice* lat, double eps, uint64_t seed, amg_gauge** out) {
    if (!lat || !out) return fail(AMG_EINVAL, "NULL argument");
    if (!std::isfinite(eps)) return fail(AMG_EINVAL, "eps must be finite");
    const GeomH& g = lat->g;
    DevBuf canon;
    if (canon.ensure((size_t)g.V * 4 * 18 * sizeof(double)) != cudaSuccess)
        return fail(AMG_ENOMEM, "gauge: device allocation failed");
    CK(launch_gauge_random(g, eps, seed, AMG_RNG_STREAM_GAUGE, canon.as<double>(), 0));
    return gauge_from_device(lat, canon.as<double>(), out);
}

amg_status amg_gauge_get(amg_gauge* G, double* host_out) {
    if (!G || !host_out) return fail(AMG_EINVAL, "NULL argument");
    const GeomH& g = G->lat->g;
    DevBuf canon;
    const size_t cb = (size_t)g.V * 4 * 18 * sizeof(double);
    CK(canon.ensure(cb));
    CK(launch_gauge_unpack64(g, G->U[0].p, canon.as<double>(), 0));
    CK(cudaMemcpy(host_out, canon.p, cb, cudaMemcpyDeviceToHost));
    return AMG_OK;
}

amg_status amg_random_normal(uint64_t seed, int stream, uint64_t start, uint64_t count, double* out, amg_stream s) {
    if (!out && count) return fail(AMG_EINVAL, "NULL output");
    if (stream < 0) return fail(AMG_EINVAL, "stream must be >= 0");
    CK(launch_random_normal(seed, (uint64_t)stream, start, count, out, (cudaStream_t)s));
    return AMG_OK;
}
void amg_gauge_destroy(amg_gauge* g) { delete g; }

amg_status amg_dirac_create(amg_gauge* g, double kappa, double csw, amg_dirac** out) {
    if (!g || !out) return fail(AMG_EINVAL, "NULL argument");
    amg_dirac* d = new amg_dirac();
    d->gauge = g;
    d->kappa = kappa;
    d->csw = csw;
    const GeomH& geo = g->lat->g;
    for (int pr = 0; pr < 4; ++pr) {
        if (d->C[pr].ensure(fine_clover_bytes(pr, geo.V)) != cudaSuccess) {
            delete d;
            return fail(AMG_ENOMEM, "clover: device allocation failed");
        }
        cudaError_t e = launch_clover_build(pr, geo, g->U[0].p, kappa, csw, d->C[pr].p, 0);
        if (e != cudaSuccess) {
            delete d;
            return fail(AMG_ECUDA, std::string("clover build: ") + cudaGetErrorString(e));
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        delete d;
        return fail(AMG_ECUDA, "clover build failed");
    }
    *out = d;
    return AMG_OK;
}
void amg_dirac_destroy(amg_dirac* d) { delete d; }

amg_status amg_dirac_get_clover(amg_dirac* d, double* host_out) {
    if (!d || !host_out) return fail(AMG_EINVAL, "NULL argument");
    const GeomH& g = d->gauge->lat->g;
    DevBuf tmp;
    size_t bytes = (size_t)g.V * 144 * sizeof(double);
    CK(tmp.ensure(bytes));
    CK(launch_clover_expand(g, d->C[0].p, tmp.as<double>(), 0));
    CK(cudaMemcpy(host_out, tmp.p, bytes, cudaMemcpyDeviceToHost));
    return AMG_OK;
}

static amg_status apply_fine_canonical(amg_dirac* d, const BlockH* sb, const void* in, void* out, int nrhs,
                                       amg_prec prec, cudaStream_t s) {
    if (!d || !in || !out || nrhs < 1) return fail(AMG_EINVAL, "bad argument");
    const GeomH& g = d->gauge->lat->g;
    if (prec == AMG_F64X && !sb) {
        CK(d->in.ensure(fine_spinor_bytes(1, g.V) * nrhs));
        CK(d->out.ensure(fine_spinor_bytes(0, g.V) * nrhs));
        CK(launch_pack_spinor(1, g, in, d->in.p, nrhs, s));
        CK(launch_dirac_mixed(g, d->gauge->U[3].p, d->C[3].p, d->in.p, d->out.p, d->kappa, nrhs, s));
        CK(launch_unpack_spinor(0, g, d->out.p, out, nrhs, s));
        return AMG_OK;
    }
    if (prec == AMG_F64D && !sb) {
        CK(d->in.ensure(fine_spinor_bytes(0, g.V) * nrhs));
        CK(d->out.ensure(fine_spinor_bytes(0, g.V) * nrhs));
        CK(launch_pack_spinor(0, g, in, d->in.p, nrhs, s));
        const size_t f32 = fine_spinor_bytes(1, g.V) * nrhs;
        CK(d->split.ensure(2 * f32));
        CK(launch_dirac_dd(g, d->gauge->U[3].p, d->C[3].p, d->gauge->U[1].p, d->C[1].p, d->in.p, d->out.p, nullptr,
                           d->kappa, nrhs, d->split.p, (char*)d->split.p + f32, s));
        CK(launch_unpack_spinor(0, g, d->out.p, out, nrhs, s));
        return AMG_OK;
    }
    if (prec < 0 || prec > 2)
        return fail(AMG_EINVAL, "prec must be AMG_F64, AMG_F32, AMG_F16 (or AMG_F64X / AMG_F64D for D)");
    size_t fb = fine_spinor_bytes(prec, g.V) * nrhs;
    CK(d->in.ensure(fb));
    CK(d->out.ensure(fb));
    CK(launch_pack_spinor(prec, g, in, d->in.p, nrhs, s));
    CK(launch_dirac(prec, g, sb, d->gauge->U[prec].p, d->C[prec].p, d->in.p, d->out.p, nullptr, d->kappa, nrhs, s));
    CK(launch_unpack_spinor(prec, g, d->out.p, out, nrhs, s));
    return AMG_OK;
}

amg_status amg_apply_D(amg_dirac* d, const void* in, void* out, int nrhs, amg_prec prec, amg_stream s) {
    return apply_fine_canonical(d, nullptr, in, out, nrhs, prec, (cudaStream_t)s);
}

amg_status amg_dirac_set_shape(amg_prec prec, int threads, int per_sm, int regs_ctas) {
    if (prec < 0 || prec > 2 || threads < 32 || threads > 256 || threads % 32 || per_sm < 1 ||
        (regs_ctas != 0 && regs_ctas != 2 && regs_ctas != 3))
        return fail(AMG_EINVAL, "bad stencil launch shape");
    dirac_set_shape(prec, threads, per_sm, regs_ctas);
    return AMG_OK;
}

amg_status amg_dirac_tune(amg_dirac* d, amg_prec prec, int* threads, int* per_sm, int* regs_ctas) {
    if (!d || prec < 0 || prec > 2) return fail(AMG_EINVAL, "prec must be AMG_F64, AMG_F32 or AMG_F16");
    const GeomH& g = d->gauge->lat->g;
    DevBuf a, b;
    CK(a.ensure(fine_spinor_bytes(prec, g.V)));
    CK(b.ensure(fine_spinor_bytes(prec, g.V)));
    CK(cudaMemset(a.p, 0, fine_spinor_bytes(prec, g.V)));
    TRY(tune_dirac_shape(d, prec, a.p, b.p));
    int t = 0, ps = 0, mb = 0;
    dirac_get_shape(prec, &t, &ps, &mb);
    if (threads) *threads = t;
    if (per_sm) *per_sm = ps;
    if (regs_ctas) *regs_ctas = mb;
    return AMG_OK;
}

amg_status amg_dirac_time(amg_dirac* d, const void* in, int nrhs, amg_prec prec, int reps, amg_stream s,
                          float* ms_per_apply) {
    if (!d || !in || !ms_per_apply || nrhs < 1 || reps < 1) return fail(AMG_EINVAL, "bad argument");
    if (prec < 0 || prec > 5 || prec == AMG_BF16)
        return fail(AMG_EINVAL, "prec must be AMG_F64, AMG_F32, AMG_F16, AMG_F64X or AMG_F64D");
    const GeomH& g = d->gauge->lat->g;
    cudaStream_t st = (cudaStream_t)s;
    const bool mixed = prec == AMG_F64X, dd = prec == AMG_F64D;
    const int pin = mixed ? 1 : dd ? 0 : prec, pout = mixed || dd ? 0 : prec;
    CK(d->in.ensure(fine_spinor_bytes(pin, g.V) * nrhs));
    CK(d->out.ensure(fine_spinor_bytes(pout, g.V) * nrhs));
    CK(launch_pack_spinor(pin, g, in, d->in.p, nrhs, st));
    if (dd) CK(d->split.ensure(2 * fine_spinor_bytes(1, g.V) * nrhs));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    amg_status rc = AMG_OK;
    cudaError_t err = cudaEventRecord(e0, st);
    for (int i = 0; err == cudaSuccess && i < reps; ++i)
        err = mixed ? launch_dirac_mixed(g, d->gauge->U[3].p, d->C[3].p, d->in.p, d->out.p, d->kappa, nrhs, st)
              : dd  ? launch_dirac_dd(g, d->gauge->U[3].p, d->C[3].p, d->gauge->U[1].p, d->C[1].p, d->in.p, d->out.p,
                                      nullptr, d->kappa, nrhs, d->split.p,
                                      (char*)d->split.p + fine_spinor_bytes(1, g.V) * nrhs, st)
                    : launch_dirac(prec, g, nullptr, d->gauge->U[prec].p, d->C[prec].p, d->in.p, d->out.p, nullptr,
                                   d->kappa, nrhs, st);
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err != cudaSuccess) rc = fail(AMG_ECUDA, cudaGetErrorString(err));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_per_apply = ms / reps;
    return rc;
}

amg_status amg_apply_Dsap(amg_dirac* d, const int block[4], const void* in, void* out, int nrhs, amg_prec prec,
                          amg_stream s) {
    if (!d || !block) return fail(AMG_EINVAL, "NULL argument");
    const GeomH& g = d->gauge->lat->g;
    BlockH b;
    for (int mu = 0; mu < 4; ++mu) {
        if (block[mu] < 1 || g.L[mu] % block[mu] != 0 || g.L[mu] / block[mu] < 2)
            return fail(AMG_EINVAL, "block must tile the lattice with >= 2 blocks per direction");
        b.b[mu] = block[mu];
    }
    return apply_fine_canonical(d, &b, in, out, nrhs, prec, (cudaStream_t)s);
}

amg_status amg_setup_from_vectors(amg_dirac* d, const amg_params* p, const double* const* vecs,
                                  amg_hierarchy** out) {
    if (!vecs || !vecs[0]) return fail(AMG_EINVAL, "vecs is NULL");
    amg_hierarchy* h = nullptr;
    TRY(hierarchy_init(d, p, out, &h));
    cudaStream_t s = 0;
    amg_status st = upload_vectors(h, vecs[0], s);
    if (st == AMG_OK) st = orthonormalise_and_galerkin(h, s);
    for (int l = 1; st == AMG_OK && l + 1 < h->p.nlevels; ++l) {
        if (!vecs[l]) st = fail(AMG_EINVAL, "test vectors missing for a coarse level");
        if (st == AMG_OK) st = upload_cvecs(h, l, vecs[l], s);
        if (st == AMG_OK) st = ortho_galerkin_c(h, l, s);
    }
    if (st == AMG_OK && cudaStreamSynchronize(s) != cudaSuccess) st = fail(AMG_ECUDA, "setup failed");
    if (st == AMG_OK) st = tune_coarse_tile(h);
    if (st == AMG_OK && h->rp == 2) h->vecs0.release();   // the solves read the half-precision copy
    if (st != AMG_OK) {
        delete h;
        return st;
    }
    *out = h;
    return AMG_OK;
}

amg_status amg_setup(amg_dirac* d, const amg_params* p, const double* const* init_vecs, amg_hierarchy** out) {
    if (!init_vecs || !init_vecs[0]) return fail(AMG_EINVAL, "init_vecs is NULL");
    amg_hierarchy* h = nullptr;
    TRY(hierarchy_init(d, p, out, &h));
    cudaStream_t s = 0;
    auto body = [&]() -> amg_status {
        TRY(upload_vectors(h, init_vecs[0], s));
        const GeomH& g = fine_geom(h);
        const int vp = h->vp;
        const size_t vb = fine_spinor_bytes(vp, g.V);
        // the test vectors go through the smoother and the cycle kSetupGroup at a time (the
        // batched kernels give each vector exactly what a call of its own gives)
        const int nv = h->p.nvec[0];
        const int G = std::min(nv, kSetupGroup);
        CK(h->tmpg.ensure(vb * G));
        // (0-a): v <- SAP(v), normalised
        for (int k = 0; k < h->p.n_init; ++k) {
            for (int i = 0; i < nv; i += G) {
                const int ng = std::min(G, nv - i);
                TRY(fine_sap(h, vp, (char*)h->vecs0.p + i * vb, h->tmpg.p, true, ng, s));
                for (int q = 0; q < ng; ++q)
                    TRY(normalise_into(h, vp, (char*)h->tmpg.p + q * vb, (char*)h->vecs0.p + (i + q) * vb, s));
            }
        }
        TRY(orthonormalise_and_galerkin(h, s));
        if (h->p.nlevels > 2) TRY(setup_coarse_level(h, 1, init_vecs, s));
        // (0-b): v <- M v with the current hierarchy, then rebuild.  Every vector of a pass goes
        // through the same M: when restriction and prolongation read vecs0 itself, the new
        // vectors are collected apart and replace vecs0 at the end of the pass; with
        // half-precision transfer vectors (vecs16, rewritten only by the rebuild) they can
        // overwrite vecs0 in place
        const bool apart = h->rp != 2;
        if (apart && h->p.n_adapt > 0) CK(h->vecs_next.ensure(vb * nv));
        if (h->p.n_adapt > 0) TRY(alloc_coarse_workspaces(h, G));
        for (int k = 0; k < h->p.n_adapt; ++k) {
            for (int i = 0; i < nv; i += G) {
                const int ng = std::min(G, nv - i);
                TRY(vcycle0(h, vp, (char*)h->vecs0.p + i * vb, h->tmpg.p, ng, s));
                for (int q = 0; q < ng; ++q) {
                    void* dst = (char*)(apart ? h->vecs_next.p : h->vecs0.p) + (i + q) * vb;
                    TRY(normalise_into(h, vp, (char*)h->tmpg.p + q * vb, dst, s));
                }
            }
            if (apart) h->vecs0.swap(h->vecs_next);
            TRY(orthonormalise_and_galerkin(h, s));
            TRY(refresh_c(h, 1, s));
        }
        h->vecs_next.release();
        h->tmpg.release();
        TRY(tune_coarse_tile(h));
        if (h->rp == 2) h->vecs0.release();   // the solves read the half-precision copy
        CK(cudaStreamSynchronize(s));
        return AMG_OK;
    };
    amg_status st = body();
    if (st != AMG_OK) {
        delete h;
        return st;
    }
    *out = h;
    return AMG_OK;
}

void amg_hierarchy_destroy(amg_hierarchy* h) { delete h; }

amg_status amg_level_info(amg_hierarchy* h, int level, int dims_out[4], int* nc_out) {
    if (!h || level < 1 || level >= h->p.nlevels) return fail(AMG_EINVAL, "bad level");
    if (dims_out)
        for (int mu = 0; mu < 4; ++mu) dims_out[mu] = h->lev[level].g.L[mu];
    if (nc_out) *nc_out = h->lev[level].nc;
    return AMG_OK;
}

amg_status amg_get_vectors(amg_hierarchy* h, int coarsening, double* host_out) {
    if (!h || !host_out || coarsening < 0 || coarsening > h->p.nlevels - 2) return fail(AMG_EINVAL, "bad argument");
    if (coarsening > 0) {
        CoarseLevel& L = h->lev[coarsening];
        const size_t n = coarse_n(L) * h->p.nvec[coarsening];
        const void* src = L.cvecs.p;
        if (L.prec != 0) {
            CK(h->canon.ensure(n * 16));
            CK(launch_convert_flat(1, 0, L.cvecs.p, h->canon.p, n, 0));
            src = h->canon.p;
        }
        CK(cudaMemcpy(host_out, src, n * 16, cudaMemcpyDeviceToHost));
        return AMG_OK;
    }
    const GeomH& g = fine_geom(h);
    const size_t cb = (size_t)g.V * 24 * sizeof(double);
    CK(h->canon.ensure(cb));
    // after a setup with half-precision transfer vectors only their copy remains (the FP32
    // vectors held exactly the rounded values)
    const bool from16 = !h->vecs0.p && h->rp == 2;
    const int vprec = from16 ? 2 : h->vp;
    const size_t vb = fine_spinor_bytes(vprec, g.V);
    for (int i = 0; i < h->p.nvec[0]; ++i) {
        const void* vi = (const char*)(from16 ? h->vecs16.p : h->vecs0.p) + i * vb;
        if (from16) {
            CK(launch_convert_spinor(2, 0, g, vi, h->fb[0].p, 1, 0));
            CK(launch_unpack_spinor(0, g, h->fb[0].p, h->canon.p, 1, 0));
        } else if (h->vp == 0) {
            CK(launch_unpack_spinor(0, g, vi, h->canon.p, 1, 0));
        } else {
            CK(launch_convert_spinor(1, 0, g, vi, h->fb[0].p, 1, 0));
            CK(launch_unpack_spinor(0, g, h->fb[0].p, h->canon.p, 1, 0));
        }
        CK(cudaMemcpy(host_out + (size_t)i * g.V * 24, h->canon.p, cb, cudaMemcpyDeviceToHost));
    }
    return AMG_OK;
}

amg_status amg_get_coarse_op(amg_hierarchy* h, int level, double* host_out) {
    if (!h || !host_out || level < 1 || level >= h->p.nlevels) return fail(AMG_EINVAL, "bad argument");
    CoarseLevel& L = h->lev[level];
    DevBuf tmp;
    size_t bytes = (size_t)L.g.V * 9 * L.nc * L.nc * 2 * sizeof(double);
    CK(tmp.ensure(bytes));
    CK(launch_coarse_op_export(L.bprec(), L.g.V, L.nc, L.B.p, tmp.as<double>(), 0));
    CK(cudaMemcpy(host_out, tmp.p, bytes, cudaMemcpyDeviceToHost));
    return AMG_OK;
}

static const uint64_t kMagic = 0x31474D41444351ull;   // "QCDAMG1"

amg_status amg_setup_save(const amg_hierarchy* hc, const char* path) {
    amg_hierarchy* h = const_cast<amg_hierarchy*>(hc);
    if (!h || !path) return fail(AMG_EINVAL, "NULL argument");
    const GeomH& g = fine_geom(h);
    // test vectors of every coarsening: fine [nvec][V][12][2], then coarse [nvec][V_l][nc][2]
    std::vector<std::vector<double>> v(h->p.nlevels - 1);
    for (int l = 0; l + 1 < h->p.nlevels; ++l) {
        const size_t per = l == 0 ? (size_t)g.V * 24 : coarse_n(h->lev[l]) * 2;
        v[l].resize(per * h->p.nvec[l]);
        TRY(amg_get_vectors(h, l, v[l].data()));
    }
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(AMG_EIO, std::string("cannot open ") + path);
    bool ok = std::fwrite(&kMagic, sizeof(kMagic), 1, f) == 1 && std::fwrite(g.L, sizeof(int), 4, f) == 4 &&
              std::fwrite(&h->p, sizeof(amg_params), 1, f) == 1;
    for (auto& vl : v) ok = ok && std::fwrite(vl.data(), sizeof(double), vl.size(), f) == vl.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? AMG_OK : fail(AMG_EIO, "write failed");
}

amg_status amg_setup_load(amg_dirac* d, const char* path, amg_hierarchy** out) {
    if (!d || !path || !out) return fail(AMG_EINVAL, "NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(AMG_EIO, std::string("cannot open ") + path);
    uint64_t magic = 0;
    int L[4];
    amg_params p;
    bool ok = std::fread(&magic, sizeof(magic), 1, f) == 1 && magic == kMagic && std::fread(L, sizeof(int), 4, f) == 4 &&
              std::fread(&p, sizeof(p), 1, f) == 1;
    const GeomH& g = d->gauge->lat->g;
    for (int mu = 0; ok && mu < 4; ++mu) ok = L[mu] == g.L[mu];
    ok = ok && p.nlevels >= 2 && p.nlevels <= AMG_MAX_LEVELS;
    std::vector<std::vector<double>> v;
    const double* vl[AMG_MAX_LEVELS] = {nullptr, nullptr, nullptr, nullptr};
    if (ok) {
        v.resize(p.nlevels - 1);
        size_t sites = g.V;
        for (int l = 0; ok && l + 1 < p.nlevels; ++l) {
            const size_t per = l == 0 ? sites * 24 : sites * 2 * (2 * p.nvec[l - 1]);
            v[l].resize(per * p.nvec[l]);
            ok = std::fread(v[l].data(), sizeof(double), v[l].size(), f) == v[l].size();
            vl[l] = v[l].data();
            for (int mu = 0; mu < 4; ++mu) sites /= (p.block[l][mu] > 0 ? p.block[l][mu] : 1);
        }
    }
    std::fclose(f);
    if (!ok) return fail(AMG_EIO, "not a checkpoint of this lattice");
    return amg_setup_from_vectors(d, &p, vl, out);
}

amg_status amg_apply_coarse(amg_hierarchy* h, int level, const void* in, void* out, int nrhs, amg_prec prec,
                            amg_stream s) {
    if (!h || !in || !out || nrhs < 1 || level < 1 || level >= h->p.nlevels) return fail(AMG_EINVAL, "bad argument");
    CoarseLevel& L = h->lev[level];
    int vprec = prec == AMG_F64 ? 0 : 1;
    cudaStream_t st = (cudaStream_t)s;
    if (prec == AMG_BF16) {
        // bfloat16 operands on the tensor cores, up to 16 right-hand sides per launch
        if (!L.opbf || !L.tci.p) return fail(AMG_EINVAL, "AMG_BF16 apply needs a bfloat16 stencil with Nc % 16 == 0");
        const size_t cv = coarse_n(L) * sizeof(float2);
        CK(h->err_flag.ensure(sizeof(int)));
        CK(cudaMemsetAsync(h->err_flag.p, 0, sizeof(int), st));
        for (int r0 = 0; r0 < nrhs; r0 += 16) {
            const int nr = std::min(16, nrhs - r0);
            CK(L.tcx.ensure(coarse_tc_pack_bytes(L.g.V, L.nc)));
            CK(launch_coarse_apply_tc(L.g, L.nc, L.tci.p, (const char*)in + r0 * cv, (char*)out + r0 * cv, nullptr, nr,
                                      L.tcx.p, h->err_flag.as<int>(), st));
        }
        int flag = 0;
        CK(cudaMemcpyAsync(&flag, h->err_flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (flag) return fail(AMG_TIMEOUT, "tensor-core coarse stencil: a wait timed out");
        return AMG_OK;
    }
    if (vprec == L.prec) {
        CK(launch_coarse_apply(L.kprec(), L.g, L.nc, nullptr, L.op(), in, out, nullptr, nrhs, st));
        return AMG_OK;
    }
    // vectors in another precision than the level's: converted through scratch that the
    // hierarchy keeps (grown when needed; stream-ordered, no synchronisation)
    size_t n = coarse_n(L) * nrhs;
    CK(h->ac_in.ensure(n * coarse_elem_bytes(L.prec)));
    CK(h->ac_out.ensure(n * coarse_elem_bytes(L.prec)));
    CK(launch_convert_flat(vprec, L.prec, in, h->ac_in.p, n, st));
    CK(launch_coarse_apply(L.kprec(), L.g, L.nc, nullptr, L.op(), h->ac_in.p, h->ac_out.p, nullptr, nrhs, st));
    CK(launch_convert_flat(L.prec, vprec, h->ac_out.p, out, n, st));
    return AMG_OK;
}

amg_status amg_coarse_time(amg_hierarchy* h, int level, const void* in, int nrhs, amg_prec prec, int reps,
                           amg_stream s, float* ms_per_apply) {
    if (!h || !in || !ms_per_apply || nrhs < 1 || reps < 1 || level < 1 || level >= h->p.nlevels)
        return fail(AMG_EINVAL, "bad argument");
    CoarseLevel& L = h->lev[level];
    const bool tc = prec == AMG_BF16;
    if (tc && (!L.opbf || !L.tci.p)) return fail(AMG_EINVAL, "AMG_BF16 needs a bfloat16 stencil with Nc % 16 == 0");
    if (!tc && ((prec == AMG_F64 ? 0 : 1) != L.prec || prec < 0 || prec > 1))
        return fail(AMG_EINVAL, "prec must be the level's vector precision or AMG_BF16");
    if (tc && nrhs > 16) return fail(AMG_EINVAL, "at most 16 right-hand sides per tensor-core launch");
    cudaStream_t st = (cudaStream_t)s;
    DevBuf out;
    CK(out.ensure(coarse_n(L) * coarse_elem_bytes(L.prec) * nrhs));
    if (tc) CK(L.tcx.ensure(coarse_tc_pack_bytes(L.g.V, L.nc)));
    CK(h->err_flag.ensure(sizeof(int)));
    CK(cudaMemsetAsync(h->err_flag.p, 0, sizeof(int), st));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    cudaError_t err = cudaEventRecord(e0, st);
    for (int i = 0; err == cudaSuccess && i < reps; ++i)
        err = tc ? launch_coarse_apply_tc(L.g, L.nc, L.tci.p, in, out.p, nullptr, nrhs, L.tcx.p, h->err_flag.as<int>(),
                                          st)
                 : launch_coarse_apply(L.kprec(), L.g, L.nc, nullptr, L.op(), in, out.p, nullptr, nrhs, st);
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return fail(AMG_ECUDA, cudaGetErrorString(err));
    int flag = 0;
    CK(cudaMemcpy(&flag, h->err_flag.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return fail(AMG_TIMEOUT, "tensor-core coarse stencil: a wait timed out");
    *ms_per_apply = ms / reps;
    return AMG_OK;
}

static amg_status transfer_common(amg_hierarchy* h, int coarsening, int nrhs, amg_prec prec) {
    if (!h || nrhs < 1) return fail(AMG_EINVAL, "bad argument");
    if (coarsening < 0 || coarsening > h->p.nlevels - 2) return fail(AMG_EINVAL, "bad coarsening");
    if (prec < 0 || prec > 3) return fail(AMG_EINVAL, "bad precision");
    if (coarsening == 0 && prec == AMG_BF16) return fail(AMG_EINVAL, "bad precision for fine fields");
    return AMG_OK;
}

// Eqs. 5-6 from coarse level l >= 1: canonical = internal coarse layout; vectors
// converted around the kernel when the caller's precision is not the level's
static amg_status coarse_transfer(amg_hierarchy* h, int l, bool restrict_dir, const void* in, void* out, int nrhs,
                                  amg_prec prec, cudaStream_t st) {
    CoarseLevel& L = h->lev[l];
    CoarseLevel& N = h->lev[l + 1];
    const int vprec = prec == AMG_F64 ? 0 : 1;
    const size_t nin = (restrict_dir ? coarse_n(L) : coarse_n(N)) * nrhs;
    const size_t nout = (restrict_dir ? coarse_n(N) : coarse_n(L)) * nrhs;
    DevBuf a, b;
    const void* src = in;
    void* dst = out;
    if (vprec != L.prec) {
        CK(a.ensure(nin * coarse_elem_bytes(L.prec)));
        CK(b.ensure(nout * coarse_elem_bytes(L.prec)));
        CK(launch_convert_flat(vprec, L.prec, in, a.p, nin, st));
        src = a.p;
        dst = b.p;
    }
    if (restrict_dir)
        CK(launch_restrict_coarse(L.prec, L.g, h->blk[l], L.nc, h->p.nvec[l], L.cvecs.p, src, dst, nrhs, st));
    else
        CK(launch_prolong_coarse(L.prec, L.g, h->blk[l], L.nc, h->p.nvec[l], L.cvecs.p, src, dst, nrhs, st));
    if (vprec != L.prec) CK(launch_convert_flat(L.prec, vprec, b.p, out, nout, st));
    CK(cudaStreamSynchronize(st));
    return AMG_OK;
}

amg_status amg_restrict(amg_hierarchy* h, int coarsening, const void* fine, void* coarse, int nrhs, amg_prec prec,
                        amg_stream s) {
    TRY(transfer_common(h, coarsening, nrhs, prec));
    if (coarsening > 0) return coarse_transfer(h, coarsening, true, fine, coarse, nrhs, prec, (cudaStream_t)s);
    const GeomH& g = fine_geom(h);
    cudaStream_t st = (cudaStream_t)s;
    int cprec = prec == AMG_F64 ? 0 : 1;
    DevBuf tmp;
    CK(tmp.ensure(fine_spinor_bytes(prec, g.V) * nrhs));
    CK(launch_pack_spinor(prec, g, fine, tmp.p, nrhs, st));
    CK(launch_restrict_fine(prec, h->rp, cprec, g, h->blk[0], h->p.nvec[0], rp_vecs(h), tmp.p, coarse, nrhs, st));
    CK(cudaStreamSynchronize(st));
    return AMG_OK;
}

amg_status amg_prolong(amg_hierarchy* h, int coarsening, const void* coarse, void* fine, int nrhs, amg_prec prec,
                       amg_stream s) {
    TRY(transfer_common(h, coarsening, nrhs, prec));
    if (coarsening > 0) return coarse_transfer(h, coarsening, false, coarse, fine, nrhs, prec, (cudaStream_t)s);
    const GeomH& g = fine_geom(h);
    cudaStream_t st = (cudaStream_t)s;
    int cprec = prec == AMG_F64 ? 0 : 1;
    DevBuf tmp;
    CK(tmp.ensure(fine_spinor_bytes(prec, g.V) * nrhs));
    CK(launch_prolong_fine(prec, h->rp, cprec, g, h->blk[0], h->p.nvec[0], rp_vecs(h), coarse, tmp.p, nrhs, st));
    CK(launch_unpack_spinor(prec, g, tmp.p, fine, nrhs, st));
    CK(cudaStreamSynchronize(st));
    return AMG_OK;
}

amg_status amg_sap(amg_hierarchy* h, const void* b, void* x, int nrhs, amg_prec prec, amg_stream s) {
    if (!h || !b || !x || nrhs < 1 || prec < 0 || prec > 2) return fail(AMG_EINVAL, "bad argument");
    const GeomH& g = fine_geom(h);
    cudaStream_t st = (cudaStream_t)s;
    if (nrhs > h->nb_cap) TRY(alloc_workspaces(h, nrhs));
    CK(h->fb[prec].ensure(fine_spinor_bytes(prec, g.V) * nrhs));
    CK(h->fx[prec].ensure(fine_spinor_bytes(prec, g.V) * nrhs));
    CK(launch_pack_spinor(prec, g, b, h->fb[prec].p, nrhs, st));
    TRY(fine_sap(h, prec, h->fb[prec].p, h->fx[prec].p, true, nrhs, st));
    CK(launch_unpack_spinor(prec, g, h->fx[prec].p, x, nrhs, st));
    CK(cudaStreamSynchronize(st));
    return AMG_OK;
}

amg_status amg_sap_coarse(amg_hierarchy* h, int level, const void* b, void* x, int nrhs, amg_prec prec,
                          amg_stream s) {
    if (!h || !b || !x || nrhs < 1 || level < 1 || level > h->p.nlevels - 2 || prec < 0 || prec > 3)
        return fail(AMG_EINVAL, "bad argument");
    CoarseLevel& L = h->lev[level];
    cudaStream_t st = (cudaStream_t)s;
    const int vprec = prec == AMG_F64 ? 0 : 1;
    const size_t n = coarse_n(L) * nrhs;
    if (vprec == L.prec) {
        TRY(coarse_sap(h, level, b, x, true, nrhs, st));
    } else {
        DevBuf a, c;
        CK(a.ensure(n * coarse_elem_bytes(L.prec)));
        CK(c.ensure(n * coarse_elem_bytes(L.prec)));
        CK(launch_convert_flat(vprec, L.prec, b, a.p, n, st));
        TRY(coarse_sap(h, level, a.p, c.p, true, nrhs, st));
        CK(launch_convert_flat(L.prec, vprec, c.p, x, n, st));
        CK(cudaStreamSynchronize(st));
        return AMG_OK;
    }
    CK(cudaStreamSynchronize(st));
    return AMG_OK;
}

amg_status amg_hierarchy_set_nn(amg_hierarchy* h, amg_nn* nn) {
    if (!h) return fail(AMG_EINVAL, "NULL hierarchy");
    if (nn && h->fp != 1) return fail(AMG_EINVAL, "the learned correction needs the FP32 smoother");
    if (nn && nn->d != h->d) return fail(AMG_EINVAL, "network and hierarchy belong to different operators");
    if (nn != h->nn) h->clear_graphs();
    h->nn = nn;
    return AMG_OK;
}

amg_status amg_precondition(amg_hierarchy* h, const double* b, double* x, amg_stream s) {
    if (!h || !b || !x) return fail(AMG_EINVAL, "bad argument");
    const GeomH& g = fine_geom(h);
    cudaStream_t st = (cudaStream_t)s;
    CK(launch_pack_spinor(0, g, b, h->ob.p, 1, st));
    TRY(precondition64(h, h->ob.p, h->oZ[0]->p, 1, st));
    if (zprec_of(h) == 0) CK(launch_unpack_spinor(0, g, h->oZ[0]->p, x, 1, st));
    else {
        CK(launch_convert_spinor(1, 0, g, h->oZ[0]->p, h->ox.p, 1, st));
        CK(launch_unpack_spinor(0, g, h->ox.p, x, 1, st));
    }
    CK(cudaStreamSynchronize(st));
    return coarse_status(h);
}

amg_status amg_solve(amg_hierarchy* h, const double* b, double* x, int nrhs, double tol, int maxit, int use_x0,
                     amg_solve_info* info, amg_stream s) {
    if (!h || !b || !x || nrhs < 1 || !(tol > 0) || maxit < 1) return fail(AMG_EINVAL, "bad argument");
    const GeomH& g = fine_geom(h);
    cudaStream_t st = (cudaStream_t)s;
    // host vectors (pinned or pageable): each batch's b is copied in on a copy stream while
    // the previous batch solves, and its x copied out while the next one solves
    auto on_host = [](const void* p) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return true;
        }
        return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
    };
    const bool host_io = on_host(b) || on_host(x);
    // the large copies go in 32 MB pieces: a copy engine serves its queue in order, and the
    // solver's small device-to-host reads on s (the Hessenberg coefficients of every step)
    // would otherwise wait behind a whole batch's vectors (tens of ms each)
    auto copy_pieces = [](void* dst, const void* src, size_t bytes, cudaStream_t cs) -> cudaError_t {
        constexpr size_t kPiece = size_t(32) << 20;
        for (size_t o = 0; o < bytes; o += kPiece) {
            cudaError_t e = cudaMemcpyAsync((char*)dst + o, (const char*)src + o, std::min(kPiece, bytes - o),
                                            cudaMemcpyDefault, cs);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    // right-hand sides solved in lockstep: up to 12, fewer if the batch's
    // workspaces (FGMRES basis, Z vectors, cycle fields) would not fit in 80%
    // of the free device memory
    int kMaxBatch = h->p.outer_solver != 0 ? 1 : 12;
    {
        const size_t f64 = fine_spinor_bytes(0, g.V), fz = fine_spinor_bytes(zprec_of(h), g.V);
        size_t per = f64 * (h->p.outer_m + 1 + 4) + fz * h->p.outer_m;
        for (int pr = 0; pr < 3; ++pr)
            if (pr == h->fp || pr == 1) per += 2 * fine_spinor_bytes(pr, g.V);
        if (host_io) per += f64;   // canonical b staging
        size_t have = 0, total = 0;
        if (cudaMemGetInfo(&have, &total) == cudaSuccess) {
            // memory the current batch capacity already holds counts as available
            size_t held = per * (size_t)h->nb_cap;
            size_t fit = (size_t)((0.8 * (double)(have + held)) / (double)per);
            if (fit < 1) fit = 1;
            if ((size_t)kMaxBatch > fit) kMaxBatch = (int)fit;
        }
    }
    amg_status worst = AMG_OK;
    amg_solve_info agg;
    std::memset(&agg, 0, sizeof(agg));
    agg.converged = 1;
    auto t_all = std::chrono::steady_clock::now();
    h->timer.reset();
    h->timer.on = info != nullptr;
    const size_t cb = fine_spinor_bytes(0, g.V);   // one canonical vector (192 B per site)
    if (host_io) {
        CK(h->io_b.ensure(cb * std::min(kMaxBatch, nrhs)));
        if (!h->io_st) CK(cudaStreamCreateWithFlags(&h->io_st, cudaStreamNonBlocking));
        for (auto& e : h->io_ev)
            if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        // work the caller queued on s before the call comes first; the first batch's b goes in
        CK(cudaEventRecord(h->io_ev[1], st));
        CK(cudaStreamWaitEvent(h->io_st, h->io_ev[1], 0));
        CK(cudaEventRecord(h->io_ev[3], h->io_st));   // the x staging starts free
        h->io_x_pending = true;
        CK(copy_pieces(h->io_b.p, b, cb * std::min(kMaxBatch, nrhs), h->io_st));
        CK(cudaEventRecord(h->io_ev[0], h->io_st));
    }
    for (int r0 = 0; r0 < nrhs; r0 += kMaxBatch) {
        const int nb = std::min(kMaxBatch, nrhs - r0);
        TRY(alloc_workspaces(h, nb));
        for (int l = 1; l < h->p.nlevels; ++l) CK(cudaMemsetAsync(h->lev[l].cs_state.p, 0, 16, st));
        std::memset(h->hstate, 0, 16 * 16);
        h->tc_cycles = 0;
        const double* br = b + (size_t)r0 * g.V * 24;
        double* xr = x + (size_t)r0 * g.V * 24;
        if (host_io) {
            // b of this batch staged (io_ev[0]); once packed, the staging takes the next batch's b
            CK(cudaStreamWaitEvent(st, h->io_ev[0], 0));
            CK(launch_pack_spinor(0, g, h->io_b.p, h->ob.p, nb, st));
            CK(cudaEventRecord(h->io_ev[1], st));
            const int r1 = r0 + nb;
            if (r1 < nrhs) {
                CK(cudaStreamWaitEvent(h->io_st, h->io_ev[1], 0));
                CK(copy_pieces(h->io_b.p, b + (size_t)r1 * g.V * 24, cb * std::min(kMaxBatch, nrhs - r1),
                               h->io_st));
                CK(cudaEventRecord(h->io_ev[0], h->io_st));
            }
            if (use_x0) {
                void* xs = h->oV[h->p.outer_m]->p;
                CK(cudaStreamWaitEvent(st, h->io_ev[3], 0));
                CK(cudaMemcpyAsync(xs, xr, cb * nb, cudaMemcpyDefault, st));
                CK(launch_pack_spinor(0, g, xs, h->ox.p, nb, st));
            } else {
                CK(cudaMemsetAsync(h->ox.p, 0, fine_spinor_bytes(0, g.V) * nb, st));
            }
        } else {
            CK(launch_pack_spinor(0, g, br, h->ob.p, nb, st));
            if (use_x0) CK(launch_pack_spinor(0, g, xr, h->ox.p, nb, st));
            else CK(cudaMemsetAsync(h->ox.p, 0, fine_spinor_bytes(0, g.V) * nb, st));
        }
        std::vector<amg_solve_info> infos;
        amg_status rs = outer_solve(h, nb, h->ob.p, h->ox.p, use_x0 != 0, tol, maxit, infos, st);
        int used_nn = (h->nn && !h->nn_off) ? 1 : 0, fell_back = 0;
        if (used_nn && (rs == AMG_NOT_CONVERGED || rs == AMG_NAN)) {
            // the FP64 residual rejects the learned correction: solve again with the plain cycle
            int prev = 0;
            for (auto& i : infos) prev = std::max(prev, i.iters);
            h->nn_off = true;
            if (use_x0 && host_io) {
                void* xs = h->oV[h->p.outer_m]->p;   // the first solve may have written it
                CK(cudaMemcpyAsync(xs, xr, cb * nb, cudaMemcpyDefault, st));
                CK(launch_pack_spinor(0, g, xs, h->ox.p, nb, st));
            } else if (use_x0) {
                CK(launch_pack_spinor(0, g, xr, h->ox.p, nb, st));
            }
            else CK(cudaMemsetAsync(h->ox.p, 0, fine_spinor_bytes(0, g.V) * nb, st));
            std::memset(h->hstate, 0, 16 * 16);
            rs = outer_solve(h, nb, h->ob.p, h->ox.p, use_x0 != 0, tol, maxit, infos, st);
            h->nn_off = false;
            for (auto& i : infos) i.iters += prev;
            used_nn = 0;
            fell_back = 1;
        }
        if (rs != AMG_OK && rs != AMG_NOT_CONVERGED) {
            if (host_io) {
                cudaStreamSynchronize(h->io_st);
                h->io_x_pending = false;
            }
            return rs;
        }
        if (host_io) {
            // x staged once the previous batch's copy-out is done; copied out while the next solves
            void* xs = h->oV[h->p.outer_m]->p;
            CK(cudaStreamWaitEvent(st, h->io_ev[3], 0));
            CK(launch_unpack_spinor(0, g, h->ox.p, xs, nb, st));
            CK(cudaEventRecord(h->io_ev[2], st));
            CK(cudaStreamWaitEvent(h->io_st, h->io_ev[2], 0));
            CK(copy_pieces(xr, xs, cb * nb, h->io_st));
            CK(cudaEventRecord(h->io_ev[3], h->io_st));
        } else {
            CK(launch_unpack_spinor(0, g, h->ox.p, xr, nb, st));
        }
        CK(cudaMemcpyAsync(h->hstate + 60, h->lev[h->p.nlevels - 1].cs_state.p, 16, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        TRY(coarse_status(h));
        h->coarse_cycles = h->hstate[63] + h->tc_cycles;
        if (rs == AMG_NOT_CONVERGED) worst = rs;
        for (auto& i : infos) {
            agg.iters = std::max(agg.iters, i.iters);
            agg.cycles = std::max(agg.cycles, i.cycles);
            agg.restarts = std::max(agg.restarts, i.restarts);
            agg.converged = agg.converged && i.converged;
            agg.true_rel_residual = std::max(agg.true_rel_residual, i.true_rel_residual);
        }
        agg.coarse_cycles += h->coarse_cycles;
        agg.batch_width = std::max(agg.batch_width, nb);
        agg.used_nn = used_nn;
        agg.nn_fallback = agg.nn_fallback || fell_back;
    }
    // the last batch's x is in the caller's memory when the call returns
    if (host_io) {
        CK(cudaStreamSynchronize(h->io_st));
        h->io_x_pending = false;
    }
    if (info) {
        double ms[PH_NPH];
        h->timer.collect(ms);
        agg.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_all).count();
        agg.ms_coarse = ms[PH_COARSE];
        agg.ms_smoother = ms[PH_SMOOTH];
        agg.ms_restrict_prolong = ms[PH_RP];
        agg.ms_products = ms[PH_PROD];
        agg.ms_orthogonalisation = ms[PH_ORTH];
        agg.ms_true_residual = ms[PH_RESID];
        agg.ms_other = agg.ms_total - ms[PH_COARSE] - ms[PH_SMOOTH] - ms[PH_RP];
        *info = agg;
    }
    h->timer.on = false;
    if (worst != AMG_OK) fail(worst, "solve did not reach the tolerance");
    return worst;
}

void amg_set_ragged_fusion(int on) { g_ragged_fused = on != 0; }

amg_status amg_solve_ragged(amg_hierarchy* const* hs, const double* const* b, double* const* x, int n, double tol,
                            int maxit, amg_solve_info* infos, amg_stream s) {
    if (!hs || !b || !x || n < 1 || !(tol > 0) || maxit < 1) return fail(AMG_EINVAL, "bad argument");
    for (int i = 0; i < n; ++i) {
        if (!hs[i] || !b[i] || !x[i]) return fail(AMG_EINVAL, "NULL hierarchy or vector");
        if (hs[i]->p.nlevels != 2) return fail(AMG_EINVAL, "ragged solves take two-grid hierarchies");
        if (hs[i]->nn) return fail(AMG_EINVAL, "ragged solves take hierarchies without a learned correction");
        if (hs[i]->p.outer_solver != 0) return fail(AMG_EINVAL, "ragged solves use the flexible GMRES outer solver");
        for (int k = 0; k < i; ++k)
            if (hs[k] == hs[i]) return fail(AMG_EINVAL, "a hierarchy appears twice in the ragged batch");
    }
    cudaStream_t user = (cudaStream_t)s;
    std::vector<RaggedProb> P(n);
    for (int i = 0; i < n; ++i) P[i].h = hs[i];
    // one launch per phase for the whole batch where the problems allow it, else a stream pool
    const bool fused = g_ragged_fused && fusable(P);
    const int ns = fused ? 1 : std::min(n, 16);
    std::vector<cudaStream_t> streams(ns, nullptr);
    cudaEvent_t ev = nullptr;
    auto t_all = std::chrono::steady_clock::now();
    auto body = [&]() -> amg_status {
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, user));
        for (auto& st : streams) {
            CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            CK(cudaStreamWaitEvent(st, ev, 0));
        }
        for (int i = 0; i < n; ++i) {
            RaggedProb& p = P[i];
            p.st = streams[i % ns];
            TRY(alloc_workspaces(p.h, 1));
            p.h->timer.on = false;
            if (fused) {
                // the fused form packs b, zeroes x and unpacks x in batch launches
                p.bcanon = b[i];
                p.xcanon = x[i];
                continue;
            }
            for (int l = 1; l < p.h->p.nlevels; ++l) CK(cudaMemsetAsync(p.h->lev[l].cs_state.p, 0, 16, p.st));
            std::memset(p.h->hstate, 0, 16 * 16);
            const GeomH& g = fine_geom(p.h);
            CK(launch_pack_spinor(0, g, b[i], p.h->ob.p, 1, p.st));
            CK(cudaMemsetAsync(p.h->ox.p, 0, fine_spinor_bytes(0, g.V), p.st));
        }
        if (fused) {
            TRY(fgmres_fused(P, streams[0], tol, maxit));
            CK(cudaStreamSynchronize(streams[0]));
            return AMG_OK;
        }
        TRY(fgmres_ragged(P, streams, tol, maxit));
        for (int i = 0; i < n; ++i) {
            RaggedProb& p = P[i];
            CK(launch_unpack_spinor(0, fine_geom(p.h), p.h->ox.p, x[i], 1, p.st));
            CK(cudaMemcpyAsync(p.h->hstate + 60, p.h->lev[p.h->p.nlevels - 1].cs_state.p, 16,
                               cudaMemcpyDeviceToHost, p.st));
        }
        for (auto st : streams) CK(cudaStreamSynchronize(st));
        for (auto& p : P) TRY(coarse_status(p.h));
        return AMG_OK;
    };
    amg_status st = body();
    for (auto sm : streams)
        if (sm) cudaStreamDestroy(sm);
    if (ev) cudaEventDestroy(ev);
    if (st != AMG_OK) return st;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_all).count();
    bool all = true;
    for (int i = 0; i < n; ++i) {
        const RhsState& r = P[i].r;
        all = all && r.conv;
        if (infos) {
            std::memset(&infos[i], 0, sizeof(amg_solve_info));
            infos[i].iters = r.iters;
            infos[i].cycles = r.iters;
            infos[i].restarts = r.restarts;
            infos[i].converged = r.conv ? 1 : 0;
            infos[i].true_rel_residual = r.bnorm == 0 ? 0.0 : r.rel;
            infos[i].ms_total = ms;
            infos[i].ms_other = ms;
            infos[i].coarse_cycles = fused ? P[i].coarse_cycles : P[i].h->hstate[63];
        }
    }
    if (!all) return fail(AMG_NOT_CONVERGED, "ragged solve: some problem did not reach the tolerance");
    return AMG_OK;
}

}  // extern "C"
