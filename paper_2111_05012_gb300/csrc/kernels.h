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

// every kernel launch of the library goes through note_launch() (a relaxed
// atomic increment); amg_launch_count() reports the running total
void note_launch();

// precision ids: 0 = F64, 1 = F32, 2 = F16, 3 = FP64 values as float hi/lo pairs (links, clover);
// coarse: 0 = F64, 1 = F32, 2 = F32 vectors with a bfloat16 operator
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
// ---- seeded inputs (inputs.cu): counter-based SplitMix64, Box-Muller, exp(i eps H) links ----
uint64_t rng_stream_key(uint64_t seed, uint64_t stream);
// complex normals start .. start+count-1 of the (seed, stream) generator, (re, im) doubles
cudaError_t launch_random_normal(uint64_t seed, uint64_t stream, uint64_t start, uint64_t count, double* out,
                                 cudaStream_t s);
// canonical double links [site][mu][3][3][2] = exp(i eps H(site, mu)) from the (seed, stream) generator
cudaError_t launch_gauge_random(const GeomH& g, double eps, uint64_t seed, uint64_t stream, double* canon,
                                cudaStream_t s);
// internal P64 links -> canonical doubles
cudaError_t launch_gauge_unpack64(const GeomH& g, const void* U64, double* canon, cudaStream_t s);
// FP64 clover build from the internal P64 gauge; writes the packed clover of prec
cudaError_t launch_clover_build(int prec, const GeomH& g, const void* U64, double kappa, double csw, void* clover,
                                cudaStream_t s);
// internal P64 clover -> [site][2][6][6][2] doubles (device)
cudaError_t launch_clover_expand(const GeomH& g, const void* C64, double* out, cudaStream_t s);

// launch shape of launch_dirac per precision (0..2): threads per CTA (a multiple of 32, <= 256),
// the grid cap in CTAs per SM, and the register budget as resident CTAs per SM (mb: 2 for FP32 /
// FP16, 128 registers; 0 or 3 = the precision's default); set by the autotuner, process-wide
void dirac_set_shape(int prec, int threads, int per_sm, int mb = 0);
void dirac_get_shape(int prec, int* threads, int* per_sm, int* mb = nullptr);
// out = D in (sap_block != NULL: hops between blocks removed); if b != NULL, out = b - D in
cudaError_t launch_dirac(int prec, const GeomH& g, const BlockH* sap_block, const void* U, const void* C,
                         const void* in, void* out, const void* b, double kappa, int nrhs, cudaStream_t s);
// out (FP64 internal) = D in (FP32 internal, exact values) with FP64-accurate double-float arithmetic;
// Udd / Cdd are the prec-3 (float hi/lo pair) link and clover fields
cudaError_t launch_dirac_mixed(const GeomH& g, const void* Udd, const void* Cdd, const void* in32, void* out64,
                               double kappa, int nrhs, cudaStream_t s);
// out (FP64 internal) = D in, or b - D in when b != NULL, for FP64 internal in: in split into
// float parts hi + lo (FP32 internal scratch fields, nrhs each), D hi in double-float arithmetic
// with the prec-3 link and clover fields, D lo in FP32 with the FP32 fields (about 46
// significant bits; the outer solver's true residual)
cudaError_t launch_dirac_dd(const GeomH& g, const void* Udd, const void* Cdd, const void* U32, const void* C32,
                            const void* in64, void* out64, const void* b64, double kappa, int nrhs, void* hi,
                            void* lo, cudaStream_t s);
// x (FP64 internal) += sum_j c[j] z[j] for k <= 20 FP32 internal fields z[j] (site-wise); pair:
// in double-float arithmetic on the FP32 pipe (about 46 significant bits) instead of FP64
cudaError_t launch_spinor_axpy_mixed(const GeomH& g, int k, const double2* c, const void* const* z, void* x,
                                     cudaStream_t s, bool pair = false);
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
// variant 3 (FP32 smoother, blocks <= 256 sites): the domain operator staged in shared memory from
// its FP16 copy (U16, C16: prec-2 fields), FP32 arithmetic and vectors; the residual b - D x uses
// the FP32 operator
cudaError_t launch_sap_half_staged16(const GeomH& g, const BlockH& bk, int colour, int nmr, int x_mode,
                                     const void* U32, const void* C32, const void* U16, const void* C16,
                                     const void* b, void* x, double kappa, int nrhs, cudaStream_t s);
// the half sweep with even-odd (Schur complement) domain solves; Ci = clover inverse of prec
// (launch_clover_invert); needs an even block extent in x and at most 512 sites per block
cudaError_t launch_sap_half_eo(int prec, const GeomH& g, const BlockH& bk, int colour, int nmr, int x_mode,
                               const void* U, const void* C, const void* Ci, const void* b, void* x, double kappa,
                               int nrhs, cudaStream_t s);
bool sap_eo_supported(const BlockH& bk);
// A^{-1} per site (two Hermitian 6x6 blocks) from the FP64 clover, stored in the clover layout of prec (0..2)
cudaError_t launch_clover_invert(int prec, const GeomH& g, const void* C64, void* out, cudaStream_t s);

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
// y = D_c x (nrhs vectors [Vc][Nc]); b != NULL: y = b - D_c x; sap_block != NULL: hops between blocks removed;
// cprec 0: FP64, 1: FP32, 2: FP32 vectors with a bfloat16 operator
cudaError_t launch_coarse_apply(int cprec, const GeomH& gc, int nc, const BlockH* sap_block, const void* B,
                                const void* in, void* out, const void* b, int nrhs, cudaStream_t s);
// ---- levels l >= 1 of a hierarchy with three or more grids (coarse_mg.cu) ----
// vprec 0: FP64, 1: FP32 (vectors, test vectors and stencils of the level).
// Vectors [V][nc] complex, test vectors [nvec][V][nc], nrhs vectors one after another.
// Eq. 5 from level l (lattice g, blocks bh) to the [Vc][2 nvec] vectors of level l+1
cudaError_t launch_restrict_coarse(int vprec, const GeomH& g, const BlockH& bh, int nc, int nvec, const void* vecs,
                                   const void* fine, void* coarse, int nrhs, cudaStream_t s);
// Eq. 6 from level l+1 back to level l
cudaError_t launch_prolong_coarse(int vprec, const GeomH& g, const BlockH& bh, int nc, int nvec, const void* vecs,
                                  const void* coarse, void* fine, int nrhs, cudaStream_t s);
// block Gram-Schmidt of the level-l test vectors per (block, chirality half); *err = 1 on rank deficiency
cudaError_t launch_orthonormalise_coarse(int vprec, const GeomH& g, const BlockH& bh, int nc, int nvec, void* vecs,
                                         int* err, cudaStream_t s);
// Eq. 7: stencil of level l+1 ([Vc][2 nvec][9][2 nvec]) from the level-l stencil B ([V][nc][9][nc]);
// computed in vprec, stored in oprec (oprec 0 with vprec 1: FP32 arithmetic widened to FP64)
cudaError_t launch_galerkin_coarse(int vprec, int oprec, const GeomH& g, const BlockH& bh, int nc, int nvec,
                                   const void* vecs, const void* B, void* Bout, cudaStream_t s);
// SAP half sweep on level l: domains of `colour`, fused residual + nmr MR steps; kprec 0 FP64,
// 1 FP32, 2 FP32 vectors with a bfloat16 stencil; x_mode as for the fine half sweep
cudaError_t launch_coarse_sap_half(int kprec, const GeomH& g, const BlockH& bh, int nc, int colour, int nmr,
                                   int x_mode, const void* B, const void* b, void* x, int nrhs, cudaStream_t s);
// persistent BiCGStab(ell) on a coarse level: one cooperative launch over every SM
// (cluster = 0) or one thread-block cluster of up to `cluster` CTAs; part and state are
// device scratch of coarse_solver_partial_bytes() / coarse_solver_state_bytes(); the first 12
// bytes of state must be zero before the launch; state word 3 accumulates the cycle count,
// word 2 is nonzero on failure (1 = barrier timeout, 2 = breakdown / non-finite)
// nb (1..coarse_solver_max_rhs()) right-hand sides in lockstep: b, x, rt, R[j], U[j] each hold nb
// vectors one after another; every stencil pass reads the operator once for all of them, and each
// right-hand side keeps its own scalars and stopping test (its iterates are those of a single solve)
size_t coarse_solver_state_bytes();
size_t coarse_solver_partial_bytes();
int coarse_solver_max_rhs();
// xgroup: coarse sites whose neighbour blocks are gathered into shared memory per step (the
// tile; 0 = as many as fit)
cudaError_t launch_coarse_bicgstab(int cprec, const GeomH& gc, int nc, const void* B, const void* b, void* x,
                                   void* rt, void* const* R, void* const* U, int ell, double tol, int maxit,
                                   void* part, void* state, int cluster, cudaStream_t s, int nb = 1,
                                   int xgroup = 0);
int coarse_solver_max_xgroup(int cprec, int nc, int nb);
// several independent single-RHS solves in one launch, one thread-block cluster per problem
// (each with its own vectors, operator, partials and state word); dev_args is device scratch of
// n * coarse_solver_desc_bytes(); all problems share cprec
struct CoarseSolveDesc {
    int cprec;
    GeomH gc;
    int nc;
    const void* B;
    const void* b;
    void* x;
    void* rt;
    void* R[5];
    void* U[5];
    int ell;
    double tol;
    int maxit;
    void* part;
    void* state;
    int xgroup;
};
size_t coarse_solver_desc_bytes();
// host_args: pinned host staging of n * coarse_solver_desc_bytes() (not rewritten before the
// copy on s is done); dev_args: device memory of the same size
cudaError_t launch_coarse_bicgstab_multi(const CoarseSolveDesc* d, int n, void* host_args, void* dev_args,
                                         cudaStream_t s);
// multi-RHS coarse stencil on the tensor cores (coarse_tc.cu): bfloat16 operands, FP32
// accumulation; needs Nc % 16 == 0 and Nc <= 64.  The operator is first copied into the
// tensor-core operand image ([V][2Nc][9Nc] bfloat16 in 8 x 8 core-matrix order) from its
// FP32 internal form; x, y, b are FP32 [nrhs][V][Nc] complex with 1 <= nrhs <= 16; xpack
// is scratch of coarse_tc_pack_bytes(V, Nc) (the packed bfloat16 vectors); *err is set
// to 1 if a wait timed out
bool coarse_tc_supported(int nc);
size_t coarse_tc_image_bytes(int V, int nc);
size_t coarse_tc_pack_bytes(int V, int nc);
cudaError_t launch_coarse_tc_image(int V, int nc, const void* B32, void* img, cudaStream_t s);
cudaError_t launch_coarse_apply_tc(const GeomH& g, int nc, const void* img, const void* x, void* y, const void* b,
                                   int nrhs, void* xpack, int* err, cudaStream_t s);
// n complex FP32 -> bfloat16 pairs (coarse operator in BF16 storage)
cudaError_t launch_complex_to_bf16(const void* in, void* out, size_t n, cudaStream_t s);
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
// y += sum_{j<k} c_j x_j (k <= 20), then in the same pass per-CTA partials of
// mode 0: |y_new|^2 (double [grid]); 1: <x_j, y_new> (double2 [k][grid]);
// 2: both, |y_new|^2 as quantity k (double2 (n2, 0), k <= 19)
// y += sum_j c_j x_j (j < k) fused with the next reduction (mode 0: |y|^2 as blas_grid()
// double partials; 1: the k dots <x_j, y>; 2: both, |y|^2 as quantity k), where the
// coefficients c_j are minus the sums of the k quantities of blas_grid() partials at csrc
// (a previous multi_dot or dot-mode reduction), summed on the device in a fixed order;
// the sums used are stored in cused[0..k) (if not NULL)
cudaError_t launch_multi_axpy_reduce_dev(int prec, int k, const double2* csrc, double2* cused, const void* const* x,
                                         void* y, size_t n, int mode, double2* partials, cudaStream_t s);
// y = x / |x| with |x|^2 the sum of the blas_grid() double partials of a norm reduction
// (y = 0 if |x| = 0); |x| is stored in *hn
cudaError_t launch_normalise(int prec, const double* norm_partials, double* hn, const void* x, void* y, size_t n,
                             cudaStream_t s);
// y = a x, a real
cudaError_t launch_scale_real(int prec, double a, const void* x, void* y, size_t n, cudaStream_t s);
// multi_dot plus |b|^2 as quantity k (double2 (n2, 0)), k <= 19
cudaError_t launch_multi_dot_norm(int prec, int k, const void* const* a, const void* b, size_t n, double2* partials,
                                  cudaStream_t s);

// ---- ragged batch: one launch per phase over per-problem descriptors ----
// One problem of a fused ragged batch (host view of the device descriptor; every pointer is
// device memory owned by the problem's hierarchy).  The fused path fixes the precisions:
// FP32 smoother, FP32 coarse vectors and operator, FP64 outer vectors; the test vectors may
// be stored in any vector precision (the same for the whole batch).
struct RaggedProbH {
    GeomH g;
    BlockH blk;
    int nvec;
    double kappa;
    const void* U32;            // FP32 links and clover
    const void* C32;
    const void* Udd;            // double-float links and clover
    const void* Cdd;
    const void* vecs;           // test vectors
    const void* v;              // V_j (FP64 internal)
    void* f32;                  // V_j in FP32
    void* f32b;                 // FP32 scratch field
    void* bc;                   // coarse right-hand side / solution, FP32 [Vc][2 nvec]
    void* xc;
    void* z;                    // Z_j = M V_j (FP32 internal)
    void* w;                    // D Z_j (FP64 internal)
    const void* basis[20];      // V_0 .. V_j
    int nbasis;                 // j + 1
    void* vnext;                // V_{j+1}
    double2* gs_part;           // Gram-Schmidt partials (2 R + ctas doubles2 at least)
    double2* gs_coef;           // 64 double2: pass-0 coefficients, pass-1 at 32, |w'| at 63
    size_t n;                   // complex entries of a fine field
    size_t R;                   // offset of the norm partials in gs_part (double2)
    const void* U64;            // FP64 links and clover (true residual)
    const void* C64;
    const void* b64;            // right-hand side, iterate, residual (FP64 internal)
    void* x64;
    void* r64;
    const void* rsrc;           // vector normalised into basis[0] (r64, or b64 while x = 0)
    double* npart;              // its norm: partials (ragged_blas_ctas(n) doubles) and value
    double* nval;
    const void* zb[20];         // x += sum_{i<k} yc[i] zb[i] (FP32 internal Z_i)
    double2 yc[20];
    int k;
    const double* canon_in;     // canonical right-hand side (packed into b64) and solution
    double* canon_out;
    int sap_nr;                 // ragged_sap_nr(block sites, largest block of the batch)
};
size_t ragged_dev_bytes();
// writes the device descriptor of h to dst (ragged_dev_bytes() bytes of host memory); -1 if invalid
int ragged_dev_fill(void* dst, const RaggedProbH& h);
// CTAs a problem takes in the site-loop phases (conversion, Arnoldi product) and in the BLAS phases
int ragged_site_ctas(int V);
int ragged_blas_ctas(size_t n);
// every launcher: d = device array of np descriptors, off = device prefix table of np + 1 CTA
// offsets for that phase (off[np] = ctas); blocks of up to 256 sites
cudaError_t launch_convert_ragged(const void* d, const int* off, int np, int ctas, cudaStream_t s);        // f32 = v
cudaError_t launch_restrict_ragged(int vprec, const void* d, const int* off, int np, int ctas, int max_vb,
                                   int max_nvec, cudaStream_t s);                                        // bc = R f32
cudaError_t launch_prolong_ragged(int vprec, const void* d, const int* off, int np, int ctas, int max_vb,
                                  int max_nvec, cudaStream_t s);                                         // z = P xc
// one SAP half sweep (x_mode 0) with right-hand side f32 and iterate z: CTAs of
// ragged_sap_threads(max_vb) threads, a problem with blocks of vb sites taking
// ceil(Vc / 2 / ragged_sap_nr(vb, max_vb)) of them
int ragged_sap_threads(int max_vb);
int ragged_sap_nr(int vb, int max_vb);
cudaError_t launch_sap_half_ragged(const void* d, const int* off, int np, int ctas, int max_vb, int colour, int nmr,
                                   cudaStream_t s);
cudaError_t launch_dirac_mixed_ragged(const void* d, const int* off, int np, int ctas, cudaStream_t s);    // w = D z
// one classical Gram-Schmidt pass against k = j + 1 basis vectors, then V_{j+1} = w' / |w'|
cudaError_t launch_gs_ragged(int k, const void* d, const int* off, int np, int ctas, int pass, cudaStream_t s);
// restart phases of a fused ragged batch (tables of the problems concerned):
// b64 = canon_in and x64 = 0; canon_out = x64; r64 = b64 - D x64 (the FP64 stencil, or with pair
// two launches: x64 split into f32 + f32b, then the pair stencil, as launch_dirac_dd); the norm
// of rsrc into nval and basis[0] = rsrc / |rsrc| (two launches); x64 += sum_i yc[i] zb[i]
cudaError_t launch_pack_ragged(const void* d, const int* off, int np, int ctas, cudaStream_t s);
cudaError_t launch_unpack_ragged(const void* d, const int* off, int np, int ctas, cudaStream_t s);
cudaError_t launch_resid_ragged(const void* d, const int* off, int np, int ctas, bool pair, cudaStream_t s);
cudaError_t launch_norm_v0_ragged(const void* d, const int* off, int np, int ctas, cudaStream_t s);
cudaError_t launch_xupdate_ragged(const void* d, const int* off, int np, int ctas, cudaStream_t s);
