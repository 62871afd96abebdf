/*
 * lqcd_amg.h -- C ABI of the GB300 adaptive-multigrid solver for the
 * Wilson-clover Dirac equation D x = b.
 *
 * Method: Kanamori, Ishikawa, Matsufuru, "Multi-grid solver for lattice QCD
 * on GPU clusters, Xeon Phi and A64FX" (arXiv:2111.05012).  Every entry point
 * names the passage that defines the operation it performs.
 *
 * Conventions shared by all calls
 * -------------------------------
 * Lattice:  dims = {Lx, Ly, Lz, Lt}; canonical site index
 *           x + Lx*(y + Ly*(z + Lz*t)); direction mu = 0..3 is x, y, z, t.
 *           Periodic in x, y, z; the fermion hop across the t boundary carries
 *           -1 when antiperiodic_t is set (Sec. 2: periodic or antiperiodic).
 * Gamma matrices: chiral basis, gamma5 = -g1 g2 g3 g4 = diag(1, 1, -1, -1).
 * Canonical fine vector (the only fine layout at the boundary):
 *           [rhs][site][spin 4][colour 3][re, im], element type double for
 *           AMG_F64, float for AMG_F32 / AMG_F16 (see amg_prec).
 * Canonical coarse vector (level l >= 1):
 *           [rhs][coarse site][Nc][re, im], Nc = 2 * nvec of the coarsening,
 *           coarse dof I = s * nvec + i (s = 0: gamma5 = +1 half, s = 1: -1).
 * Gauge field (host, double): [site][mu][row 3][col 3][re, im].
 *
 * Ownership: handles are created and freed by the library (children before
 * parents).  Host arrays passed to *_create / setup calls are copied.  Vector
 * pointers given to apply / restrict / prolong / solve calls are caller-owned
 * DEVICE pointers, borrowed for the duration of the call; work is enqueued on
 * the given stream (NULL = the legacy default stream).
 *
 * Errors: every call returns an amg_status; nothing aborts, nothing throws
 * across the ABI.  amg_last_error() returns a message for the last failure on
 * the calling thread.
 */
#ifndef LQCD_AMG_H
#define LQCD_AMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int amg_status;
#define AMG_OK 0
#define AMG_EINVAL 1            /* bad argument (sizes, blocking, precision, NULL) */
#define AMG_ENOMEM 2            /* device or host allocation failed */
#define AMG_ECUDA 3             /* a CUDA call failed; see amg_last_error() */
#define AMG_NOT_CONVERGED 4     /* iteration cap reached; best iterate returned */
#define AMG_NAN 5               /* non-finite residual / breakdown */
#define AMG_TIMEOUT 6           /* a bounded device-side wait gave up */
#define AMG_EIO 7               /* file read/write failed (checkpoints) */

typedef enum {
    AMG_F64 = 0,   /* double storage and arithmetic */
    AMG_F32 = 1,   /* float storage and arithmetic */
    AMG_F16 = 2,   /* fine fields stored as half with a per-site float scale, float arithmetic */
    AMG_BF16 = 3,  /* coarse operator stored as bfloat16, float accumulation */
    AMG_F64X = 4,  /* amg_apply_D only: float input (taken as exact), double output, FP64-accurate
                      double-float arithmetic with FP64 links and clover (the outer solver's Arnoldi
                      product for vectors produced by the FP32 preconditioner) */
    AMG_F64D = 5   /* amg_apply_D only: double input and output, every input value split into a float
                      pair, the same double-float arithmetic (about 46 significant bits; the outer
                      solver's true residual b - D x when the smoother is not FP64) */
} amg_prec;

#define AMG_MAX_LEVELS 4

typedef struct amg_lattice amg_lattice;
typedef struct amg_gauge amg_gauge;
typedef struct amg_dirac amg_dirac;
typedef struct amg_hierarchy amg_hierarchy;
typedef struct amg_nn amg_nn;
typedef struct CUstream_st* amg_stream;   /* = cudaStream_t */

/* Multigrid parameters (Sec. 3; numbers in brackets are defaults from
 * amg_params_default).  Level 0 is the fine lattice; coarsening l maps level
 * l to level l+1 with block[l] and nvec[l]. */
typedef struct {
    int nlevels;                        /* number of grids, 2..AMG_MAX_LEVELS [2] */
    int block[AMG_MAX_LEVELS - 1][4];   /* block dims per coarsening, {bx, by, bz, bt} [4,4,4,4] */
    int nvec[AMG_MAX_LEVELS - 1];       /* test vectors per coarsening [24] */
    int n_init;                         /* setup (0-a): SAP applications per test vector [3] */
    int n_adapt;                        /* setup (0-b): adaptive passes v <- M v [2] */
    int sap_iters;                      /* SAP iterations n of the Sec. 3 listing [4] */
    int mr_iters;                       /* inner-domain minimal-residual steps [6] */
    double coarse_tol;                  /* coarsest solve, relative residual [1e-2] */
    int coarse_maxit;                   /* coarsest solve, BiCGStab(l) cycles [200] */
    int coarse_ell;                     /* l of BiCGStab(l), 1..4 [2] */
    int inter_m;                        /* intermediate levels: flexible GMRES(m) [8] */
    double inter_tol;                   /* intermediate levels: relative tolerance [1e-1] */
    int inter_maxit;                    /* intermediate levels: max steps [8] */
    int outer_m;                        /* outer flexible GMRES restart length [16] */
    int prec_smoother;                  /* fine D / SAP / R / P precision: AMG_F64, AMG_F32, AMG_F16 [AMG_F32] */
    int prec_coarse;                    /* coarse operators above the coarsest: AMG_F64, AMG_F32, AMG_BF16 [AMG_F32] */
    int prec_coarsest;                  /* coarsest-level solve: AMG_F64, AMG_F32, or AMG_BF16 =
                                           FP32 vectors and arithmetic with the coarse operator
                                           stored in bfloat16 (half the bytes per stencil sweep)
                                           [AMG_F32] */
    int sap_variant;                    /* SAP kernel: -1 autotune at setup (times the variants for one
                                           right-hand side and for a batch, keeps the fastest of each),
                                           0 operator read from global memory, 1 operator staged in shared
                                           memory (FP32/FP16, blocks <= 256 sites; two right-hand sides
                                           per CTA in a batch), 2 as 0 but two right-hand sides of a batch
                                           per CTA sharing the operator in L1 (FP32/FP16, <= 256 sites),
                                           3 FP32 smoother with the operator staged in shared memory from
                                           its FP16 copy (<= 256 sites; residual with the FP32 operator)
                                           [-1] */
    int outer_solver;                   /* 0: flexible GMRES(outer_m) [0]; 1: the paper's BiCGStab with
                                           flexible preconditioning (Sec. 3), one right-hand side at a
                                           time; 2: the paper's comparison solver MBiCGs (Sec. 5,
                                           Table 1): the same flexible BiCGStab preconditioned by
                                           BiCGStab(coarse_ell) on the fine operator itself in the
                                           smoother precision (FP32 or FP64), from zero to
                                           mbicgs_tol or mbicgs_maxit cycles, no multigrid; all stop
                                           on the FP64 true residual */
    int prec_vectors;                   /* fine test vectors as read by restriction and prolongation
                                           (Eqs. 5, 6): AMG_F16 stores them in half precision with a
                                           per-site scale (about half the bytes of each transfer); the
                                           setup rounds the orthonormalised vectors to it and builds the
                                           Galerkin operator (Eq. 7) from the rounded ones, so R, P and
                                           D_c stay consistent.  Any other value keeps the setup's
                                           precision (FP64 with an FP64 smoother, else FP32).  AMG_F16
                                           needs an FP32 or FP16 smoother [AMG_F32] */
    double mbicgs_tol;                  /* MBiCGs inner solve: relative residual [1e-4] */
    int mbicgs_maxit;                   /* MBiCGs inner solve: BiCGStab(l) cycles [50] */
    int sap_eo;                         /* 1: the fine-level SAP domain solves in even-odd (Schur
                                           complement) form -- mr_iters minimal-residual steps on
                                           S = A_ee - H_eo A_oo^{-1} H_oe over the even sites of the
                                           domain, then z_o = A_oo^{-1}(r_o - H_oe z_e) exactly (H the
                                           in-domain hops, A = 1 + F); needs an even block extent in
                                           x; the clover inverse is built once per operator and
                                           precision.  Not in the paper (an addition beside the SAP
                                           listing of Sec. 3).  0: the paper's MR on D_SAP [0] */
    int coarse_tc;                      /* 1: a batch of 2..16 right-hand sides on a coarsest level stored
                                           in bfloat16 (prec_coarsest = AMG_BF16, Nc % 16 == 0) runs its
                                           coarse BiCGStab(l) in lockstep with every stencil pass on the
                                           tensor cores (bfloat16 operands including the vectors, FP32
                                           accumulation); 0: the persistent SIMT solver for every batch
                                           (four right-hand sides per launch) [0] */
    int resid_pair;                     /* outer solver's true residual b - D x: 0 the FP64 stencil;
                                           1 (smoother not FP64) x split into float parts and D in the
                                           double-float pair arithmetic of the Arnoldi product on the
                                           FP32 pipe, about 46 significant bits [0] */
} amg_params;

typedef struct {
    int iters;                  /* outer flexible GMRES steps (= preconditioner applications) */
    int restarts;
    int converged;              /* 1 if ||b - D x|| / ||b|| <= tol in FP64 */
    double true_rel_residual;   /* FP64 ||b - D x|| / ||b|| recomputed at exit */
    double ms_total;            /* wall time of the call */
    double ms_coarse;           /* time in coarse solves (the phase split of Table 1) */
    double ms_smoother;         /* time in SAP */
    double ms_restrict_prolong; /* time in restriction + prolongation */
    double ms_other;            /* everything else (outer Krylov, residuals, conversions) */
    int coarse_cycles;          /* total BiCGStab(l) cycles on the coarsest level */
    int used_nn;                /* 1 if the learned correction was part of the preconditioner */
    int nn_fallback;            /* 1 if the solve was redone with the plain cycle */
    int cycles;                 /* preconditioner applications (= iters for flexible GMRES, two per
                                   iteration for flexible BiCGStab); largest over a batch */
    double ms_products;         /* part of ms_other: the outer solver's products D z (FP64-accurate) */
    double ms_orthogonalisation;/* part of ms_other: FP64 Gram-Schmidt and normalisation (GPU time) */
    double ms_true_residual;    /* part of ms_other: FP64 b - D x at restarts and exit */
    int batch_width;            /* right-hand sides per lockstep batch (largest batch of the call) */
} amg_solve_info;

/* Message of the last failed call on this thread ("" if none). */
const char* amg_last_error(void);

/* Number of CUDA kernels this library has run since it was loaded (all
 * threads, all devices; a running total, never reset): direct launches, plus
 * every kernel of a captured CUDA graph each time the graph is replayed.  No
 * counterpart in the paper: lets a caller count the kernels behind a call. */
unsigned long long amg_launch_count(void);

/* Fill p with the defaults listed above. */
void amg_params_default(amg_params* p);

/* ---- lattice and fields (Sec. 2) ------------------------------------- */

/* A 4D lattice.  dims must be >= 2 in every direction.  Fails with
 * AMG_EINVAL otherwise. */
amg_status amg_lattice_create(const int dims[4], int antiperiodic_t, amg_lattice** out);
void amg_lattice_destroy(amg_lattice* lat);

/* Gauge field U_mu(x) (Eq. 1) from host memory, canonical gauge layout,
 * V*4*9 complex doubles.  Copied to the device (FP64 master, plus FP32/FP16
 * two-row forms on demand). */
amg_status amg_gauge_create(amg_lattice* lat, const double* U_host, amg_gauge** out);
void amg_gauge_destroy(amg_gauge* g);

/* Seeded synthetic inputs.  The paper's experiments (Sec. 5) use gauge
 * ensembles that are not distributed with it; the workloads of this library
 * stand in for them with U_mu(x) = exp(i eps H), H = (A + A^dag)/2 minus its
 * trace / 3, A a 3x3 complex matrix with N(0, 1) real and imaginary parts.
 * Random numbers: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) in counter
 * mode -- word n of stream (seed, id) is mix64(key + (n + 1) * G) with
 * G = 0x9E3779B97F4A7C15 and key = mix64(seed * G + id); a word w gives the
 * double ((w >> 11) + 1) * 2^-53 in (0, 1]; complex normal m is the
 * Box-Muller pair of words 2m and 2m + 1: sqrt(-2 ln u0) (cos, sin)(2 pi u1).
 * Generated on the device; every value is a pure function of (seed, id, m),
 * so a host implementation of the same definition reproduces it to the
 * rounding of ln, sqrt, cos and sin. */
#define AMG_RNG_STREAM_GAUGE 1     /* link entries: complex normal 9 (4 site + mu) + row-major entry */
#define AMG_RNG_STREAM_RHS 2       /* Gaussian right-hand sides (seed + 1000 by convention) */
#define AMG_RNG_STREAM_TESTVEC 3   /* initial test vectors (seed + 2000 + 1000 level by convention) */
#define AMG_RNG_STREAM_NN 6        /* training errors e0 of the learned preconditioner */

/* Gauge field U_mu(x) = exp(i eps H_mu(x)) with A drawn from stream
 * (seed, AMG_RNG_STREAM_GAUGE); the exponential is evaluated in FP64 from the
 * eigenvalues of eps H (unitary, det 1 to rounding).  Same handle as
 * amg_gauge_create, without a host copy of the field.  AMG_EINVAL for a
 * NULL argument or non-finite eps, AMG_ENOMEM / AMG_ECUDA on device failure. */
amg_status amg_gauge_random(amg_lattice* lat, double eps, uint64_t seed, amg_gauge** out);

/* Copy the FP64 links of g to host memory in the canonical gauge layout
 * (V*4*9 complex doubles, caller-owned). */
amg_status amg_gauge_get(amg_gauge* g, double* host_out);

/* Complex normals start .. start+count-1 of stream (seed, stream) written to
 * the device array out as (re, im) doubles (2*count doubles, caller-owned),
 * on stream s.  A canonical fine field of volume V is count = 12 V; field k
 * of a stream starts at start = 12 V k.  AMG_EINVAL for a NULL output with
 * count > 0 or a negative stream id. */
amg_status amg_random_normal(uint64_t seed, int stream, uint64_t start, uint64_t count, double* out, amg_stream s);

/* Wilson-clover operator of Eq. 1 with hopping parameter kappa and clover
 * coefficient csw.  Builds the clover term F(x) on the device in FP64 from
 * the links: F = -kappa csw sum_{mu<nu} sigma_munu F_munu, F_munu the
 * traceless anti-Hermitian part of the four-leaf clover divided by 8i,
 * sigma_munu = [gamma_mu, gamma_nu]/(2i).  In the chiral basis 1 + F is two
 * 6x6 Hermitian blocks per site. */
amg_status amg_dirac_create(amg_gauge* g, double kappa, double csw, amg_dirac** out);
void amg_dirac_destroy(amg_dirac* d);

/* Copy 1 + F(x) to host memory as [site][chirality 2][6][6][re, im] doubles
 * (row/col index = (spin - 2*chirality)*3 + colour). */
amg_status amg_dirac_get_clover(amg_dirac* d, double* host_out);

/* out = D in (Eq. 1) for nrhs canonical fine vectors (device pointers).
 * prec selects the storage/arithmetic of D and the element type of in/out:
 * double for AMG_F64 and AMG_F64D, float for AMG_F32 / AMG_F16, float in and
 * double out for AMG_F64X.  in and out must not alias. */
amg_status amg_apply_D(amg_dirac* d, const void* in, void* out, int nrhs, amg_prec prec, amg_stream s);

/* out = D in, exactly as amg_apply_D, but without allocating device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate, e.g. a process whose device memory is fully reserved by a
 * caching allocator or a latency-critical loop that must not pay the
 * device-wide synchronisation of cudaMalloc/cudaFree.  amg_apply_D converts
 * the canonical vectors to and from the internal layout in two work fields
 * the library allocates on first use; this variant keeps those two fields in
 * one static device array of 24 MiB (12 MiB each) that every GPU loading the
 * library holds until exit.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) once for that device and keeps it for
 * the life of the process; make that first call before any stream capture.
 * Resetting the device (cudaDeviceReset) or otherwise recreating its primary
 * context after that first call is not supported: the array may then live at
 * another address.  Every call shares the array, so calls that
 * overlap on the GPU (different streams, or host threads) race: serialise
 * them.  nrhs * fine_field_bytes(prec) must be <= 12 MiB, where a field is
 * 192 (AMG_F64), 96 (AMG_F32) or 52 (AMG_F16) bytes per site; larger calls
 * fail with AMG_EINVAL.  in, out: canonical device vectors as for
 * amg_apply_D (element type double for AMG_F64, float otherwise). */
amg_status amg_apply_D_noalloc(amg_dirac* d, const void* in, void* out, int nrhs, amg_prec prec, amg_stream s);

/* Autotune the launch shape of the fine stencil in precision prec (AMG_F64,
 * AMG_F32, AMG_F16) on d's lattice: CTA size and grid cap, and for FP32 / FP16
 * the register budget (2 resident CTAs per SM, 128 registers, against the
 * default).  The choice is process-wide and used by every later stencil
 * launch of that precision (amg_setup runs the same tuner for the precisions
 * a solve uses).  Outputs (may be NULL): threads per CTA, grid cap in CTAs
 * per SM, register budget as resident CTAs per SM (0 = the default).
 * Synchronises the device.  No counterpart in the paper. */
amg_status amg_dirac_tune(amg_dirac* d, amg_prec prec, int* threads, int* per_sm, int* regs_ctas);

/* Set the stencil's launch shape for prec by hand (process-wide, as amg_dirac_tune
 * leaves it): threads per CTA (a multiple of 32, at most 256), grid cap in CTAs
 * per SM (>= 1), register budget as resident CTAs per SM (0 or 3 = the
 * precision's default, 2 = 128 registers; FP64 ignores it).  AMG_EINVAL otherwise. */
amg_status amg_dirac_set_shape(amg_prec prec, int threads, int per_sm, int regs_ctas);

/* Timing of the Eq. 1 stencil alone: packs the canonical input `in` (nrhs
 * fields, element type as for amg_apply_D) into the library's internal layout
 * once, then applies D to it `reps` times on stream s, bracketed by CUDA
 * events, and writes the mean milliseconds per application to *ms_per_apply.
 * The result field is discarded.  Synchronises s.  prec AMG_F64 / AMG_F32 /
 * AMG_F16, or AMG_F64X (float input, the FP64-accurate double-float kernel
 * of the outer solver's Arnoldi product).  No counterpart in the paper: the
 * kernel-only time that the roofline of the stencil is computed from. */
amg_status amg_dirac_time(amg_dirac* d, const void* in, int nrhs, amg_prec prec, int reps, amg_stream s,
                          float* ms_per_apply);

/* out = D_SAP in: D with every hop between different blocks of size block[4]
 * switched off (Sec. 3, SAP paragraph).  block must tile the lattice with at
 * least two blocks per direction. */
amg_status amg_apply_Dsap(amg_dirac* d, const int block[4], const void* in, void* out, int nrhs,
                          amg_prec prec, amg_stream s);

/* ---- multigrid hierarchy (Sec. 3 step 0) ------------------------------ */

/* Adaptive setup, steps (0-a) and (0-b) of Sec. 3: the init vectors are
 * smoothed by n_init SAP applications, block-orthonormalised in FP64 per
 * (domain, chirality) by Gram-Schmidt applied twice, the Galerkin coarse
 * operator D_c = <I|D|J> (Eq. 7) is built, then n_adapt passes v <- M v
 * follow.  init_vecs[l] is a host array of nvec[l] canonical vectors of
 * level l (doubles: fine [site][spin][colour][re, im], coarse
 * [site][Nc][re, im]), one array for every level 0..nlevels-2, each in host
 * or device memory (copied with cudaMemcpyDefault); the random numbers of
 * the setup are these inputs (amg_random_normal draws them on the device).  With three or more grids, level
 * l >= 1 is set up the same way with its own SAP and cycle, right after its
 * stencil is first built; every later change of level l's stencil rebuilds
 * the stencils below it from their unchanged vectors.
 * Fails with AMG_EINVAL on a bad blocking or a rank-deficient domain. */
amg_status amg_setup(amg_dirac* d, const amg_params* p, const double* const* init_vecs,
                     amg_hierarchy** out);

/* Hierarchy from given test vectors without smoothing: orthonormalise and
 * build the Galerkin operators (Eqs. 5-7) level by level.  Used by
 * checkpoint loading and for exact parity tests of the construction. */
amg_status amg_setup_from_vectors(amg_dirac* d, const amg_params* p, const double* const* vecs,
                                  amg_hierarchy** out);
void amg_hierarchy_destroy(amg_hierarchy* h);

/* Coarse lattice dims and Nc of level l (1 <= l < nlevels). */
amg_status amg_level_info(amg_hierarchy* h, int level, int dims_out[4], int* nc_out);

/* Orthonormalised test vectors of coarsening l as canonical level-l vectors
 * (host doubles, nvec[l] of them). */
amg_status amg_get_vectors(amg_hierarchy* h, int coarsening, double* host_out);

/* Coarse operator of level l >= 1 as host doubles [site][d 9][Nc][Nc][re, im]
 * with d = 0 self, 1+mu the block coupling X to X+mu, 5+mu to X-mu, so that
 * y(X) = sum_d B[X][d] x(X + d) (the 9-point stencil of Eq. 7).  Returned as
 * computed (FP64 or FP32), before any bfloat16 storage rounding. */
amg_status amg_get_coarse_op(amg_hierarchy* h, int level, double* host_out);

/* Save / load the test vectors and parameters of a hierarchy (the setup is
 * reused for many right-hand sides, Sec. 3).  Loading rebuilds the coarse
 * operators from the stored vectors with amg_setup_from_vectors. */
amg_status amg_setup_save(const amg_hierarchy* h, const char* path);
amg_status amg_setup_load(amg_dirac* d, const char* path, amg_hierarchy** out);

/* ---- transfer and coarse operators (Eqs. 5-7) -------------------------- */

/* y = D_c x on level l >= 1 (the 9-point stencil), nrhs canonical coarse
 * vectors (element type double for AMG_F64, float otherwise).  AMG_F64 /
 * AMG_F32: the operator is applied as the level stores it (bfloat16 entries
 * with FP32 accumulation when the level was built with a bfloat16 stencil).
 * AMG_BF16: the tensor-core path for levels with a bfloat16 stencil and
 * Nc % 16 == 0 (AMG_EINVAL otherwise): the vectors are rounded to bfloat16
 * and each coarse site's rows are one dense contraction over up to 16
 * right-hand sides at a time (tcgen05 MMA, FP32 accumulation in tensor
 * memory); AMG_TIMEOUT if a bounded wait in the kernel gave up. */
amg_status amg_apply_coarse(amg_hierarchy* h, int level, const void* in, void* out, int nrhs,
                            amg_prec prec, amg_stream s);

/* Timing of the coarse stencil alone: applies it `reps` times to the nrhs
 * canonical coarse vectors `in` on stream s (results discarded), bracketed by
 * CUDA events, and writes the mean milliseconds per application.  prec: the
 * level's vector precision (AMG_F64 / AMG_F32: the SIMT stencil) or AMG_BF16
 * (the tensor-core path, nrhs <= 16).  Synchronises s.  No counterpart in the
 * paper: the kernel-only time behind the roofline of the coarse stencil. */
amg_status amg_coarse_time(amg_hierarchy* h, int level, const void* in, int nrhs, amg_prec prec, int reps,
                           amg_stream s, float* ms_per_apply);

/* Eq. 5: coarse(I) = <I|fine> from level `coarsening` to coarsening+1.
 * fine is canonical at that level (a fine field for coarsening 0, a coarse
 * vector [site][Nc] for coarsening >= 1); element type from prec as above. */
amg_status amg_restrict(amg_hierarchy* h, int coarsening, const void* fine, void* coarse, int nrhs,
                        amg_prec prec, amg_stream s);

/* Eq. 6: fine = sum_I coarse(I) |I>. */
amg_status amg_prolong(amg_hierarchy* h, int coarsening, const void* coarse, void* fine, int nrhs,
                       amg_prec prec, amg_stream s);

/* x = SAP(b) on the fine lattice (Sec. 3 listing: x = 0, r = b, n times
 * {x += M_e r; r = b - Dx; x += M_o r; r = b - Dx}, M = mr_iters minimal
 * residual steps per domain), in the smoother precision, for nrhs canonical
 * vectors one after another (the batched kernels of a lockstep solve). */
amg_status amg_sap(amg_hierarchy* h, const void* b, void* x, int nrhs, amg_prec prec, amg_stream s);

/* x = SAP(b) on coarse level 1 <= level <= nlevels-2 (three or more grids):
 * the same listing with the level's blocks as domains and D_SAP the level's
 * 9-point stencil without the hops between blocks.  nrhs canonical coarse
 * vectors; prec AMG_F64 (double) or AMG_F32 / AMG_BF16 (float). */
amg_status amg_sap_coarse(amg_hierarchy* h, int level, const void* b, void* x, int nrhs, amg_prec prec,
                          amg_stream s);

/* x = M b: one application of the multigrid preconditioner (Sec. 3 steps
 * (1) and (2)).  Canonical double vectors. */
amg_status amg_precondition(amg_hierarchy* h, const double* b, double* x, amg_stream s);

/* Ragged batch: n independent problems (each its own lattice, operator and
 * two-grid hierarchy; no hierarchy twice, none with a learned correction)
 * solved to ||b_i - D_i x_i|| <= tol ||b_i|| in FP64 from x_i = 0, as
 * amg_solve does for one right-hand side.  The problems' outer flexible
 * GMRES steps run in lockstep with one host synchronisation per step for all
 * of them.  Fused form (the default, when every problem has an FP32
 * smoother, FP32 coarse vectors, the same coarse operator storage, test-vector
 * precision, sap_iters and mr_iters, blocks of at most 256 sites and
 * outer_m <= 19): each phase of an Arnoldi step -- the FP64 -> FP32 copy of
 * V_j, restriction, the coarse BiCGStab(l) (one thread-block cluster per
 * problem), prolongation, each SAP half sweep, the Arnoldi product and the
 * Gram-Schmidt pass -- is one kernel launch over a table of per-problem
 * descriptors, whatever n is.  Otherwise (or after amg_set_ragged_fusion(0))
 * each problem's step runs on a pool of up to 16 streams, captured into a
 * CUDA graph on first use (kept in the hierarchy until its workspaces grow
 * or its learned correction changes) and replayed.  b[i], x[i]: canonical
 * double device vectors of problem i.  infos (may be NULL) receives n
 * records.  Ordered after earlier work on stream s; synchronises.  No
 * counterpart in the paper (a batch of independent solves of Sec. 3). */
amg_status amg_solve_ragged(amg_hierarchy* const* h, const double* const* b, double* const* x, int n, double tol,
                            int maxit, amg_solve_info* infos, amg_stream s);
/* Process-wide switch of amg_solve_ragged between the fused form (on = 1, the
 * default) and the stream pool (on = 0). */
void amg_set_ragged_fusion(int on);

/* ---- learned preconditioner -------------------------------------------- */
/* The paper's preconditioner slot (Sec. 3 steps (1)-(2)) extended by a
 * gauge-equivariant network of parallel-transport convolution layers
 *   out^a(x) = sum_b sum_d W_d^{ab} (T_d in^b)(x),
 * T_0 = 1, (T_{+mu} f)(x) = U_mu(x) f(x+mu), (T_{-mu} f)(x) = U_mu(x-mu)^dag f(x-mu)
 * (fermion boundary phase as in Eq. 1), d = 0 self, 1+mu forward, 5+mu
 * backward; W_d^{ab} a complex 4x4 spin matrix.  Weights are kept in FP32 on
 * the host, applied in bfloat16 with FP32 accumulation. */

/* Network with nlayers linear layers, channels[0] = channels[nlayers] = 1,
 * 1..4 channels per layer.  weights: host floats, layer after layer,
 * [C_out][C_in][9][4][4][re, im] (copied). */
amg_status amg_nn_create(amg_dirac* d, int nlayers, const int* channels, const float* weights, amg_nn** out);
void amg_nn_destroy(amg_nn* nn);

/* Current weights in the layout of amg_nn_create; effective != 0 returns the
 * bfloat16-rounded values the kernels apply. */
amg_status amg_nn_get_weights(amg_nn* nn, int effective, float* host_out);

/* One layer: in = C_in canonical float fields, out = C_out fields (device). */
amg_status amg_nn_layer_forward(amg_nn* nn, int layer, const float* in, float* out, amg_stream s);

/* Backward of one layer for an output gradient grad_out (dL/d conj(out)):
 * grad_in (may be NULL) = L^dag grad_out (C_in fields, device), grad_w (host
 * doubles, may be NULL) = dL/d conj(W) in the weight layout
 * (d/dRe W = 2 Re, d/dIm W = 2 Im).  Synchronises the stream. */
amg_status amg_nn_layer_backward(amg_nn* nn, int layer, const float* in, const float* grad_out, float* grad_in,
                                 double* grad_w, amg_stream s);

/* out = N(in) for one canonical float field. */
amg_status amg_nn_apply(amg_nn* nn, const float* in, float* out, amg_stream s);

/* One Adam step (lr, betas 0.9/0.999) on npairs (residual, error) pairs
 * (canonical float fields, device) for the loss mean ||N(r) - e||^2/||e||^2;
 * loss_out (may be NULL) receives the batch loss before the step. */
amg_status amg_nn_train_step(amg_nn* nn, const float* r, const float* e, int npairs, double lr, double* loss_out,
                             amg_stream s);

/* Training run of amg_learned_train. */
typedef struct {
    int npairs;      /* (residual, error) pairs generated and trained on [4096] */
    int batch;       /* pairs per Adam step; npairs / batch steps are taken [16] */
    double lr;       /* Adam learning rate (betas 0.9 / 0.999, eps 1e-8) [1e-3] */
    uint64_t seed;   /* e0 of pair k: canonical field k of stream (seed, AMG_RNG_STREAM_NN) [5] */
} amg_train_params;

/* Fill p with the defaults listed above. */
void amg_train_params_default(amg_train_params* p);

/* Train nn on (residual, error) pairs that the solver itself makes on its own
 * gauge field, all on the device: for pair k, e0 = Gaussian field k of stream
 * (seed, AMG_RNG_STREAM_NN), e = e0 - M D e0 (the error one application of the
 * multigrid preconditioner M of Sec. 3 leaves, with D and M as in
 * amg_apply_D / amg_precondition in FP64), r = D e; the pairs (r, e) are
 * rounded to FP32 and every `batch` of them makes one amg_nn_train_step.
 * losses (host, may be NULL) receives npairs / batch batch losses, in order.
 * nn must have been created on the hierarchy's operator.  Synchronises the
 * stream.  The paper has no learned preconditioner; this is the task's
 * extension of the preconditioner slot of Sec. 3 (see amg_hierarchy_set_nn
 * for its use in a solve). */
amg_status amg_learned_train(amg_hierarchy* h, amg_nn* nn, const amg_train_params* p, double* losses,
                             amg_stream s);

/* Use the network inside the solve's preconditioner (NULL removes it):
 * z = M v + N(v - D M v) with the FP32 cycle M.  If a solve with it misses
 * the tolerance or breaks down, amg_solve redoes it with the plain cycle
 * (info->nn_fallback = 1).  Requires prec_smoother = AMG_F32. */
amg_status amg_hierarchy_set_nn(amg_hierarchy* h, amg_nn* nn);

/* ---- solve ------------------------------------------------------------- */

/* Solve D x = b for nrhs canonical double vectors with flexible GMRES(outer_m)
 * preconditioned by the multigrid cycle, until the FP64 true residual
 * ||b - D x|| / ||b|| <= tol (recomputed at every restart and at exit) or
 * maxit outer steps.  Up to 12 right-hand sides are solved in lockstep: one
 * batched cycle (restriction, coarse solves, prolongation, SAP over all of
 * them) and one batched Arnoldi product per step.  The Arnoldi basis is
 * orthogonalised by classical Gram-Schmidt in FP64 with the coefficients
 * summed on the device (one host synchronisation per step), with a second
 * pass wherever eps ||w|| / ||w'|| would exceed 1e-9.  With outer_solver = 1
 * the paper's flexible BiCGStab runs instead, one right-hand side at a
 * time.  b and x may be device memory, or host memory (pinned, or pageable):
 * then each batch's b is copied in on the hierarchy's copy stream while the
 * previous batch solves, and its x copied out while the next batch solves
 * (device staging of one batch of each; pinned memory lets the copies
 * overlap the solves); the call returns with x in host memory.  x is an input initial
 * guess if use_x0 != 0, else overwritten.  info (may be NULL) receives, over
 * all right-hand sides, the largest iteration count and true residual, the
 * summed phase times and whether all converged.  Returns AMG_NOT_CONVERGED
 * if any rhs misses tol. */
amg_status amg_solve(amg_hierarchy* h, const double* b, double* x, int nrhs, double tol, int maxit,
                     int use_x0, amg_solve_info* info, amg_stream s);

#ifdef __cplusplus
}
#endif
#endif /* LQCD_AMG_H */
