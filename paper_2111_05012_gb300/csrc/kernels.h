// Host-callable launchers of the library's CUDA kernels (no device types).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

struct GeomH {
    int L[4];
    int V;
    int antiperiodic;
};
struct BlockH {
    int b[4];
};

// precision ids: 0 = F64, 1 = F32, 2 = F16, 3 = FP64 values as float hi/lo pairs (links, clover);
// coarse: 0 = F64, 1 = F32
size_t fine_spinor_bytes(int prec, int V);
size_t fine_gauge_bytes(int prec, int V);
size_t fine_clover_bytes(int prec, int V);

// canonical [site][12][re,im] (double for prec 0, float otherwise) <-> internal
cudaError_t launch_pack_spinor(int prec, const GeomH& g, const void* canon, void* internal, int nrhs, cudaStream_t s);
cudaError_t launch_unpack_spinor(int prec, const GeomH& g, const void* internal, void* canon, int nrhs, cudaStream_t s);
// internal precision conversion (nrhs fields)
cudaError_t launch_convert_spinor(int prec_in, int prec_out, const GeomH& g, const void* in, void* out, int nrhs,
                                  cudaStream_t s);
// canonical double gauge [site][mu][3][3][2] (device) -> internal of prec
cudaError_t launch_gauge_convert(int prec, const GeomH& g, const double* canon, void* internal, cudaStream_t s);
// FP64 clover build from the internal P64 gauge; writes the packed clover of prec
cudaError_t launch_clover_build(int prec, const GeomH& g, const void* U64, double kappa, double csw, void* clover,
                                cudaStream_t s);
// internal P64 clover -> [site][2][6][6][2] doubles (device)
cudaError_t launch_clover_expand(const GeomH& g, const void* C64, double* out, cudaStream_t s);

// out = D in (sap_block != NULL: hops between blocks removed); if b != NULL, out = b - D in
cudaError_t launch_dirac(int prec, const GeomH& g, const BlockH* sap_block, const void* U, const void* C,
                         const void* in, void* out, const void* b, double kappa, int nrhs, cudaStream_t s);
// out (FP64 internal) = D in (FP32 internal, exact values) with FP64-accurate double-float arithmetic;
// Udd / Cdd are the prec-3 (float hi/lo pair) link and clover fields
cudaError_t launch_dirac_mixed(const GeomH& g, const void* Udd, const void* Cdd, const void* in32, void* out64,
                               double kappa, int nrhs, cudaStream_t s);
// x (FP64 internal) += sum_j c[j] z[j] for k <= 20 FP32 internal fields z[j] (site-wise)
cudaError_t launch_spinor_axpy_mixed(const GeomH& g, int k, const double2* c, const void* const* z, void* x,
                                     cudaStream_t s);
// one SAP half sweep on the domains of one colour (fused residual + MR):
//   r = b - D x on the domain, z = MR_nmr(D_SAP, r), x += z
//   x_mode 0: x holds the iterate; 1: x is zero everywhere; 2: x is zero on the active domains
cudaError_t launch_sap_half(int prec, const GeomH& g, const BlockH& bk, int colour, int nmr, int x_mode,
                            const void* U, const void* C, const void* b, void* x, double kappa, cudaStream_t s);

// variant 0: operator read from global memory in every MR step (all precisions);
// variant 1: domain operator staged in shared memory (FP32 / FP16, blocks <= 256 sites)
cudaError_t launch_sap_half_variant(int variant, int prec, const GeomH& g, const BlockH& bk, int colour, int nmr,
                                    int x_mode, const void* U, const void* C, const void* b, void* x, double kappa,
                                    int nrhs, cudaStream_t s);
bool sap_staged_supported(int prec, const BlockH& bk);

// ---- transfer (fine level 0 -> 1) ----
// fprec: field precision (0/1/2), vprec: test-vector precision (0/1), cprec: coarse precision (0/1)
// nrhs fields / coarse vectors one after another (blockIdx.y = right-hand side)
cudaError_t launch_restrict_fine(int fprec, int vprec, int cprec, const GeomH& g, const BlockH& bk, int nvec,
                                 const void* vecs, const void* fine, void* coarse, int nrhs, cudaStream_t s);
cudaError_t launch_prolong_fine(int fprec, int vprec, int cprec, const GeomH& g, const BlockH& bk, int nvec,
                                const void* vecs, const void* coarse, void* fine, int nrhs, cudaStream_t s);
// block Gram-Schmidt (twice) in FP64 on nvec internal fine vectors; *err_flag set to 1 on rank deficiency
cudaError_t launch_orthonormalise_fine(int vprec, const GeomH& g, const BlockH& bk, int nvec, void* vecs,
                                       int* err_flag, cudaStream_t s);
// Galerkin coarse stencil from the fine operator; B layout [Vc][Nc][9][Nc] of cprec
cudaError_t launch_galerkin_fine(int vprec, int cprec, const GeomH& g, const BlockH& bk, int nvec, const void* vecs,
                                 const void* U, const void* C, double kappa, void* B, cudaStream_t s);

// ---- coarse level ----
// y = D_c x (nrhs vectors [Vc][Nc]); b != NULL: y = b - D_c x; sap_block != NULL: hops between blocks removed
cudaError_t launch_coarse_apply(int cprec, const GeomH& gc, int nc, const BlockH* sap_block, const void* B,
                                const void* in, void* out, const void* b, int nrhs, cudaStream_t s);
// coarse SAP half sweep (fused residual + MR) on level >= 1
cudaError_t launch_coarse_sap_half(int cprec, const GeomH& gc, int nc, const BlockH& bk, int colour, int nmr,
                                   int x_zero, const void* B, const void* b, void* x, cudaStream_t s);
// coarse-level transfer (level l >= 1 -> l+1): fields [Vc][nc], vectors [nvec][Vc][nc]
cudaError_t launch_restrict_coarse(int prec, const GeomH& gc, int nc, const BlockH& bk, int nvec, const void* vecs,
                                   const void* fine, void* coarse, int cprec_out, cudaStream_t s);
cudaError_t launch_prolong_coarse(int prec, const GeomH& gc, int nc, const BlockH& bk, int nvec, const void* vecs,
                                  const void* coarse, int cprec_in, void* fine, cudaStream_t s);
cudaError_t launch_orthonormalise_coarse(int prec, const GeomH& gc, int nc, const BlockH& bk, int nvec, void* vecs,
                                         int* err_flag, cudaStream_t s);
cudaError_t launch_galerkin_coarse(int prec, int cprec_out, const GeomH& gc, int nc, const BlockH& bk, int nvec,
                                   const void* vecs, const void* B, void* Bout, cudaStream_t s);
// persistent BiCGStab(ell) on a coarse level (one cooperative launch); part and state are
// device scratch of coarse_solver_partial_bytes() / coarse_solver_state_bytes(); the first 12
// bytes of state must be zero before the launch; state word 3 accumulates the cycle count,
// word 2 is nonzero on failure (1 = barrier timeout, 2 = breakdown / non-finite)
size_t coarse_solver_state_bytes();
size_t coarse_solver_partial_bytes();
cudaError_t launch_coarse_bicgstab(int cprec, const GeomH& gc, int nc, const void* B, const void* b, void* x,
                                   void* rt, void* const* R, void* const* U, int ell, double tol, int maxit,
                                   void* part, void* state, cudaStream_t s);
// coarse op layout change: internal [Vc][Nc][9][Nc] -> canonical [Vc][9][Nc][Nc] doubles
cudaError_t launch_coarse_op_export(int cprec, int Vc, int nc, const void* B, double* out, cudaStream_t s);
// precision change of flat complex arrays (n complex numbers); prec 0 = double2, 1 = float2
cudaError_t launch_convert_flat(int prec_in, int prec_out, const void* in, void* out, size_t n, cudaStream_t s);

// ---- BLAS-1 on flat complex arrays (prec 0 = double2, 1 = float2) ----
// partial sums: per-CTA double2 partials written to `partials` (k dots of a[i] with b, grid CTAs each)
int blas_grid();
cudaError_t launch_multi_dot(int prec, int k, const void* const* a, const void* b, size_t n, double2* partials,
                             cudaStream_t s);
cudaError_t launch_norm2(int prec, const void* a, size_t n, double* partials, cudaStream_t s);
// y = alpha * x + beta * y  (alpha, beta complex)
cudaError_t launch_axpby(int prec, double2 alpha, const void* x, double2 beta, void* y, size_t n, cudaStream_t s);
// y += sum_j c[j] * x[j]  (k vectors, coefficients host-side)
cudaError_t launch_multi_axpy(int prec, int k, const double2* c, const void* const* x, void* y, size_t n,
                              cudaStream_t s);
