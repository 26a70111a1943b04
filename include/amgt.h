/*
 * amgt.h -- C ABI of the GB300 (sm_103a) angular-multigrid DG transport library.
 *
 * The library solves the steady mono-energetic linear Boltzmann equation
 *     Omega . grad phi + sigma_t phi = Q,  phi = phi_in on inflow boundaries
 * (Lathouwers & Perko, arXiv 2010.04559, Sec. 2, Eq. LBE) discretised by
 * discontinuous Galerkin in space (Q1 on axis-aligned quads/hexes) and in
 * angle (spherical patches, Const or Lin basis; Sec. 2.1-2.3), with the
 * Legendre-expanded scatter source of Sec. 4.2 and the angular multigrid
 * preconditioner of Sec. 4 (Fig. lmg) inside restarted GMRES or BiCGStab.
 *
 * Conventions shared by every call
 * --------------------------------
 * Cells: c = ix + nx*(iy + ny*iz).  Spatial nodes of a cell: i = a + 2b + 4c
 * for the corner (a, b, c) in {0,1}^dim, x fastest; s = 2^dim nodes.
 * Angular mesh: octant o = 4*bx + 2*by + bz (bit 1 = negative axis sign),
 * vertices (sx e_x, sy e_y, sz e_z); a patch (a, b, c) splits into
 * (a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca) with ab = (a+b)/|a+b|;
 * patches are numbered depth first.  Lin function m of a patch is the nodal
 * function of its vertex m; Const has one function.  a = 3 (Lin) or 1.
 * Vectors: psi[Nsdof][Nadof] row major, sdof = c*s + i, adof = q*a + m
 * (Eq. Expansion).  Multigrid level k = 0 is the finest angular mesh T_L,
 * level k is T_{L-k}.
 *
 * Ownership: set_* calls copy their inputs; the context owns every table and
 * workspace; the caller owns every buffer it passes.  Device pointers passed
 * to amgt_op_* are read/written on the context's stream, asynchronously.
 * Errors: every call returns an amgt_status and never throws across the
 * ABI; amgt_last_error() gives the message of the last failing call.  A
 * context is not thread safe; use one per host thread / stream.
 */
#ifndef AMGT_H
#define AMGT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amgt_ctx amgt_ctx;

typedef enum {
  AMGT_OK = 0,
  AMGT_ERR_ARG = -1,            /* invalid argument or call order            */
  AMGT_ERR_CUDA = -2,           /* a CUDA runtime call failed                */
  AMGT_ERR_NOMEM = -3,          /* device allocation failed                  */
  AMGT_ERR_NOT_CONVERGED = -4,  /* GMRES reached maxit above tol             */
  AMGT_ERR_BREAKDOWN = -5,      /* Krylov breakdown without convergence      */
  AMGT_ERR_NAN = -6,            /* NaN/Inf met in a residual                 */
  AMGT_ERR_DEVICE_TIMEOUT = -7, /* a bounded device-side wait gave up        */
  AMGT_ERR_STATE = -8,          /* problem not fully specified               */
  AMGT_ERR_UNSUPPORTED = -9     /* configuration outside the kernels' scope  */
} amgt_status;

/* element types of device buffers passed to amgt_op_* */
#define AMGT_F64 0      /* double                                              */
#define AMGT_F32 1      /* float                                               */
#define AMGT_F32_BF16TC 2 /* float in/out, scatter contraction on BF16 tensor
                             cores with FP32 accumulation (amgt_op_scatter)   */
#define AMGT_F64_SPLIT 3  /* double in/out, scatter contraction to FP64
                             accuracy from BF16 tensor-core products: the
                             operands are cut into integer digit slices whose
                             products the FP32 accumulator holds exactly
                             (error-free splitting of Ozaki et al., 2012),
                             summed in FP64; falls back to the FP64 SIMT
                             contraction where the angular size is below 64,
                             not a multiple of 8, or tcgen05 is absent       */
#define AMGT_F32_TC3 4    /* float in/out, scatter contraction to FP32 accuracy
                             on FP16 tensor cores: each row of sigma_s N x is
                             scaled by a power of two and cut into a high and
                             a low FP16 part (S_f likewise), and the three
                             products hi S_hi + lo S_hi + hi S_lo run as one
                             GEMM over the concatenated inner dimension with
                             FP32 accumulation (relative error ~2^-21); same
                             fallback as AMGT_F64_SPLIT, to the FP32 SIMT
                             contraction                                      */

/* preconditioners and precision modes of amgt_solve */
#define AMGT_PREC_NONE 0
#define AMGT_PREC_SWEEP 1     /* M^-1 = L^-1, Krylov-accelerated source iteration (Sec. 3) */
#define AMGT_PREC_MG 2        /* linear V-cycle of Fig. lmg (Sec. 4)              */
#define AMGT_MODE_F64 0       /* everything in FP64                               */
#define AMGT_MODE_MIXED 1     /* FP64 GMRES as iterative refinement around an FP32
                                 flexible GMRES (FP32-accurate operator, its
                                 scatter as AMGT_F32_TC3) whose multigrid
                                 preconditioner runs FP32 sweeps/transfers and the
                                 BF16 tensor-core scatter (FP32 accumulation)     */

typedef struct amgt_options {
  double tol;          /* stop when ||b - A x||_2 / ||b||_2 < tol (Sec. 5.1)   */
  int restart;         /* GMRES restart length m (<= 0: 20; at most 30, the
                          Krylov workspace; larger values run GMRES(30))    */
  int maxit;           /* cap on Krylov iterations (all cycles; <= 0: 1000)    */
  int precond;         /* AMGT_PREC_*                                          */
  int mode;            /* AMGT_MODE_*                                          */
  int device_ptrs;     /* 1: x0/psi/phi of amgt_solve are device pointers      */
  double inner_tol;    /* mixed mode: relative tol of each inner FP32 solve;
                          0: adaptive, each inner solve aims at the outer tol:
                          0.3 tol / (current relres), within [3e-5, 1e-2],
                          and stops after 2 restart cycles at most          */
  int inner_maxit;     /* mixed mode: cap per inner solve (<= 0: 200)          */
  int krylov;          /* AMGT_KRYLOV_GMRES (restarted GMRES(restart)) or
                          AMGT_KRYLOV_BICGSTAB (the paper's method, Sec. 3);
                          in mixed mode it is the inner FP32 solver          */
} amgt_options;
#define AMGT_KRYLOV_GMRES 0
#define AMGT_KRYLOV_BICGSTAB 1

#define AMGT_MAX_HIST 1024
typedef struct amgt_stats {
  int iterations;          /* Krylov iterations (inner ones in mixed mode)     */
  int outer_iterations;    /* refinement steps (mixed) / restarts (FP64)       */
  double relres;           /* final true ||b - A x|| / ||b||, FP64             */
  double seconds;          /* wall time of the solve                           */
  int nhist;               /* entries of hist                                  */
  double hist[AMGT_MAX_HIST]; /* estimated relative residual per iteration     */
} amgt_stats;

/* ---- context -------------------------------------------------------------- */
/* Creates a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (may be NULL for the legacy default stream); every call issues its work on
 * it.  Returns AMGT_OK and *out, or an error. */
int amgt_create(amgt_ctx** out, int device, void* cuda_stream);
void amgt_destroy(amgt_ctx* ctx);
/* Message of the last failing call on this context (never NULL). */
const char* amgt_last_error(const amgt_ctx* ctx);
int amgt_set_stream(amgt_ctx* ctx, void* cuda_stream);
/* Number of CUDA kernels the library has launched in this process so far
 * (all contexts).  Host-side counter; no device work. */
int amgt_query_launches(int64_t* count);
/* Device time of the library's main kernels, from CUDA events that the
 * library records on its stream around each launch while the tuning key
 * AMGT_TUNE_KERNEL_TIMERS is 1 (no events otherwise).  `kernel` is one of
 * AMGT_KT_*; *ms receives the summed duration and *launches the number of
 * timed launches since the last reset (reset != 0 clears them after
 * reading).  Waits for the recorded events. */
#define AMGT_KT_SWEEP 0        /* transport sweep L^-1                         */
#define AMGT_KT_APPLY_L 1      /* L x                                          */
#define AMGT_KT_SCATTER_PREP 2 /* FP32 -> BF16 operand pass of the TC scatter  */
#define AMGT_KT_SCATTER_TC 3   /* tcgen05 BF16 scatter GEMM                    */
#define AMGT_KT_SCATTER_F32 4  /* FP32 scatter contractions (SIMT)             */
#define AMGT_KT_COARSE_GS 5    /* coarse Gauss-Seidel kernel                   */
#define AMGT_KT_SCATTER_F64 6  /* FP64 scatter contractions (SIMT)             */
#define AMGT_KT_SPLIT_TC 7     /* tcgen05 GEMMs of the split FP64 scatter      */
#define AMGT_KT_SPLIT_AUX 8    /* digit slicing and FP64 accumulation of it    */
#define AMGT_KT_TC3 9          /* tcgen05 FP16 GEMM of the AMGT_F32_TC3 scatter */
#define AMGT_KT_TC3_PREP 10    /* its FP32 -> FP16 hi/lo operand pass          */
#define AMGT_KT_COUNT 11
int amgt_query_kernel_time(amgt_ctx* ctx, int kernel, int reset, double* ms, int64_t* launches);
/* As amgt_query_kernel_time, and *work (may be NULL) receives the summed
 * algorithmic work of the timed launches, counted by the library from each
 * launch's shapes: bytes for the memory-bound classes (SWEEP: read b and
 * write psi; APPLY_L: read x, write y, and read y when it accumulates;
 * SCATTER_PREP: 4 B read + 2 B written per unknown; TC3_PREP: 4 + 6 B;
 * SPLIT_AUX: the digit slicing's and the FP64 accumulation's reads and
 * writes), flop for the contractions (SCATTER_TC, SPLIT_TC: 2 M N K of the
 * GEMM; TC3: 2 M N (3K); SCATTER_F32/F64: 2 M N^2 dense or 4 M N nmom in
 * moment form; COARSE_GS: 2 flop per multiply-add of the sequential
 * per-patch block solves, (2 s a nm + s a^2 + s^2 a + (s a)^2) per cell,
 * patch and sweep).  reset clears all three counters. */
int amgt_query_kernel_stats(amgt_ctx* ctx, int kernel, int reset, double* ms, int64_t* launches,
                            double* work);
/* Blocks until all work issued on the context's stream has finished; returns
 * AMGT_ERR_DEVICE_TIMEOUT if a device-side bounded wait gave up since the
 * last check. */
int amgt_sync(amgt_ctx* ctx);

/* ---- problem statement (Sec. 2, Eq. LBE; Sec. 2.1; Sec. 4.2; Sec. 5) ----- */
/* Axis-aligned box [lo, hi] cut into ncell[0] x ncell[1] (x ncell[2]) equal
 * cells; dim = 2 (slab infinite and uniform in z) or 3. */
int amgt_set_mesh_cartesian(amgt_ctx* ctx, int dim, const int64_t ncell[3],
                            const double lo[3], const double hi[3]);
/* Per-cell sigma_t[C] and sigma_s[C] (= sigma_{s,0}) on host memory, and the
 * Legendre moment shapes f[nmat][N+1] (row-major) of nmat materials, the
 * material of cell c being mat_id[c]: sigma_{s,n}(c) = sigma_s[c] *
 * f[mat_id[c]][n] (f[m][0] = 1; Sec. 4.2, Eq. for Q).  mat_id may be NULL
 * when nmat = 1 (one shape for every cell).  The scatter kernel is
 * sum_n (2n+1)/(4 pi) sigma_{s,n} P_n(Omega.Omega').  With several shapes the
 * scatter runs in moment form (each cell's moments scaled by its shape) on
 * the SIMT GEMM and the coarse Gauss-Seidel in its per-patch form; the dense,
 * tensor-core and split forms need one shape.  Requires the mesh.
 * AMGT_ERR_ARG for sigma_t <= 0, sigma_s < 0, non-finite values, mat_id out
 * of [0, nmat) or f[m][0] != 1. */
int amgt_set_materials(amgt_ctx* ctx, const double* sigma_t, const double* sigma_s,
                       const int32_t* mat_id, int nmat, int N, const double* f);
/* Uniform angular mesh of the given level (8*4^level patches; Sec. 2.1).
 * basis: 0 Const, 1 Lin (Sec. 2.2). */
int amgt_set_angular_uniform(amgt_ctx* ctx, int basis, int level);
/* Mesh refined about `axis` by the bands 0.97/0.9/0.8/0.6 of Sec. 5.4: an
 * element is split while its level is below the band of the largest
 * Omega.axis over its vertices (lmax, lmax-1, ..., floored at 0). */
int amgt_set_angular_aniso(amgt_ctx* ctx, int basis, const double axis[3], int lmax);
/* k-level V(nu_pre, nu_post) cycle on T_L..T_{L-k+1} (Fig. lmg).  Nr[j] is
 * the scatter order used on level j (Sec. 4.3; Nr[0] normally N).  The
 * coarsest level is solved by coarse_sweeps block Gauss-Seidel sweeps
 * (Sec. 4.2; 0: no coarse correction).  nlevels = 1 keeps only the finest
 * mesh, and the cycle is then the Gauss-Seidel sweeps alone. */
int amgt_set_multigrid(amgt_ctx* ctx, int nlevels, const int* Nr, int nu_pre,
                       int nu_post, int coarse_sweeps);
/* Isotropic volumetric source: q[C] scalar emission density, Q = q/(4 pi). */
int amgt_set_source_iso(amgt_ctx* ctx, const double* q);
/* Boundary face f = 2*axis + side (side 1 = high): kind 0 vacuum, kind 1
 * isotropic inflow of angular flux params[0], kind 2 a normally incident
 * pencil beam of strength S = params[0] (particles per unit face area),
 * uniform over the face, kind 3 a pencil beam of any inward direction over a
 * rectangle of the face: params = {S, Omega_b[3], u0, u1, v0, v1}, Omega_b
 * (normalised by the library) with Omega_b . n < 0, the beam covering the
 * face points whose tangential coordinates (the face's other axes in
 * increasing order) lie in [u0, u1] x [v0, v1] (in 2D [u0, u1]; v0, v1 are
 * read but unused), clipped to the face (Sec. 5.4: the cube with a boundary
 * source on a square of its face).  A beam psi_b = S delta(Omega - Omega_b)
 * is taken in the DG weak form: the patches whose closed spherical triangle
 * holds Omega_b share the Dirac mass by the fraction of an infinitesimal cap
 * around Omega_b lying in each (1 inside, 1/2 on an edge, interior angle /
 * 2 pi at a vertex: 1/4 each at the octahedron vertex of kind 2), and patch
 * q receives S |Omega_b . n| share_q Psi_m(Omega_b) times the integral of the
 * spatial basis function over the beam's part of the face.  params is read
 * at the call (1 value for kinds 1 and 2, 8 for kind 3); AMGT_ERR_ARG for a
 * face or kind out of range, a non-finite value, a zero or outward beam
 * direction or an empty range. */
int amgt_set_boundary(amgt_ctx* ctx, int face, int kind, const double* params);
/* Kernel tuning knobs (results do not depend on them beyond rounding):
 *   AMGT_TUNE_GS_KERNEL   0 auto, 1 per-patch coarse Gauss-Seidel kernel,
 *                         2 direction-blocked kernel, one warp per cell,
 *                         3 direction-blocked kernel, one thread group per
 *                         cell with the tables in shared memory when they fit
 *                         (else as 2), 4 the thread-group form over the whole
 *                         GPU: one block per cell, cooperative launch, bounded
 *                         grid barrier between wavefront levels, 5 (FP32) the
 *                         thread-block form with the contractions on tensor
 *                         cores (split-TF32 MMAs, 8 cells per block), 6 the
 *                         row-pipelined form: each block owns whole rows of
 *                         cells (lines along x) and exchanges face values
 *                         with the blocks of the neighbouring rows through
 *                         tagged words, no barrier between wavefront levels
 *                         (cooperative launch; a face wait gives up after
 *                         2 s and reports AMGT_ERR_DEVICE_TIMEOUT at the next
 *                         amgt_sync); 0 picks 6, else 3, else 2, else 1 (2 to
 *                         6 use precomputed block lower-triangular inverses:
 *                         the same iteration up to rounding)
 *   AMGT_TUNE_SWEEP_GROUP patches per sweep thread block (0 = auto)
 *   AMGT_TUNE_SWEEP_STAGES depth of the 2D sweep's copy pipeline (0 = auto,
 *                         2, 3, 4 or 6 levels)
 *   AMGT_TUNE_GS_GRID_BLOCKS blocks of the whole-GPU and of the row-pipelined
 *                         Gauss-Seidel (0 = auto; fewer blocks than rows give
 *                         each block several rows)
 *   AMGT_TUNE_GS_CLUSTER  cluster size of the cluster Gauss-Seidel kernels
 *                         (0 = largest available, else 1, 2, 4, 8 or 16)
 *   AMGT_TUNE_KERNEL_TIMERS 1: time the main kernels with CUDA events (see
 *                         amgt_query_kernel_time), 0: off (default)
 *   AMGT_TUNE_GRAPHS      1: amgt_solve applies the multigrid preconditioner
 *                         by replaying a CUDA graph of the V-cycle captured on
 *                         its first use (input and output through two fixed
 *                         device buffers); 0: direct launches (default).
 *                         Ignored while the kernel timers are on and on
 *                         the default stream (which cannot be captured).
 *   AMGT_TUNE_FP64_SCATTER the FP64 scatter contraction: 0 auto (the mixed
 *                         solve's FP64 refinement residuals in the split
 *                         form of AMGT_F64_SPLIT, every other FP64 scatter
 *                         on the FP64 SIMT GEMM), 1 FP64 SIMT everywhere,
 *                         2 split form everywhere (FP64 solves too)
 *   AMGT_TUNE_SPLIT_ROWS  rows of psi per pass of the split form (0 = auto:
 *                         as many as keep its digit slices within ~8 GB;
 *                         else rounded up to a multiple of 128)
 *   AMGT_TUNE_SWEEP_KERNEL the 2D sweep: 0 auto (2 where a block holds at
 *                         least two patches in FP32 or four in FP64, else
 *                         1), 1 level-synchronous row
 *                         kernel (one block barrier per wavefront level),
 *                         2 warp-pipelined kernel (Lin basis, 2, 4 or 8
 *                         patches per block: each warp runs its own skewed
 *                         wavefront over its rows and hands the boundary
 *                         row to the next warp through a shared ring with a
 *                         step counter; a wait gives up after 2 s and
 *                         reports AMGT_ERR_DEVICE_TIMEOUT at the next
 *                         amgt_sync); cases outside 2's scope run 1.  In
 *                         3D, 0 and 2 run every direction and patch in one
 *                         cooperative launch, level by level with a grid
 *                         barrier between wavefront levels (a barrier that
 *                         waits 2 s reports AMGT_ERR_DEVICE_TIMEOUT at the
 *                         next amgt_sync), and 1 the level kernel with one
 *                         block per direction and patch group.
 *   AMGT_TUNE_F32_SCATTER the FP32 scatter of the mixed solve's inner
 *                         operator: 0 auto (the FP16 three-product tensor-
 *                         core form of AMGT_F32_TC3 where it applies), 1 the
 *                         FP32 SIMT contraction
 *   AMGT_TUNE_COARSE_F64  the coarsest-level Gauss-Seidel solve of the FP32
 *                         V-cycle (mixed solves, AMGT_F32 cycles): 0 in FP32
 *                         (default), 1 in FP64 (the right-hand side converted
 *                         to FP64, the FP64 sweeps, the result rounded back)
 *   AMGT_TUNE_GS_FORM     the row-pipelined coarse Gauss-Seidel's scattering
 *                         source: 0 auto (with one moment shape in use, the
 *                         dense form where the angular unknowns are fewer
 *                         than twice the moments plus a direction's unknowns,
 *                         and in FP32 also where its register kernel applies:
 *                         2D Lin patches, at most 96 angular unknowns and two
 *                         materials), 1 the moment form (flux moments kept
 *                         per cell), 2 the dense form S_f x_c where it applies;
 *                         takes effect at the next set-up (the context is
 *                         rebuilt before its next use)
 *   AMGT_TUNE_TEST_SWEEP_HOLD for tests of the failure path only: 1 makes
 *                         the warp-pipelined 2D sweep's first warp of each
 *                         block withhold its progress counter and every wait
 *                         of that kernel give up after 10 ms instead of 2 s,
 *                         so the launch ends early with psi undefined and the
 *                         next amgt_sync returns AMGT_ERR_DEVICE_TIMEOUT (the
 *                         context stays usable); 0 (default) normal */
#define AMGT_TUNE_GS_KERNEL 1
#define AMGT_TUNE_SWEEP_GROUP 2
#define AMGT_TUNE_SWEEP_STAGES 3
#define AMGT_TUNE_GS_GRID_BLOCKS 4
#define AMGT_TUNE_GS_CLUSTER 5
#define AMGT_TUNE_KERNEL_TIMERS 6
#define AMGT_TUNE_GRAPHS 7
#define AMGT_TUNE_FP64_SCATTER 8
#define AMGT_TUNE_SPLIT_ROWS 9
#define AMGT_TUNE_SWEEP_KERNEL 10
#define AMGT_TUNE_F32_SCATTER 11
#define AMGT_TUNE_TEST_SWEEP_HOLD 12
#define AMGT_TUNE_COARSE_F64 13
#define AMGT_TUNE_GS_FORM 14
int amgt_set_tuning(amgt_ctx* ctx, int key, int value);
/* Times the sweep's patches per block and copy depth (what bit 0) and the
 * coarse Gauss-Seidel kernel (what bit 1) on this context's own hierarchy
 * (CUDA events on its stream, FP32) and keeps the fastest; results are
 * cached per problem shape for the process.  choice (may be NULL) receives
 * {patches per block, copy stages, Gauss-Seidel kernel, 1 if cached}. */
int amgt_autotune(amgt_ctx* ctx, int what, int* choice);
/* Sizes of level k of the hierarchy. */
int amgt_query_sizes(const amgt_ctx* ctx, int level, int64_t* nsdof, int64_t* nadof);

/* Solves (L - S) psi = f to opt->tol (Sec. 3, Sec. 5.1).  psi [Nsdof][Nadof]
 * and phi [Nsdof] (scalar flux, may be NULL) receive the result; x0 may be
 * NULL (zero initial guess) and may equal psi (a warm start in place, e.g.
 * to resume a solve).  Pointers are host memory unless opt->device_ptrs.
 * st may be NULL. */
int amgt_solve(amgt_ctx* ctx, const amgt_options* opt, const double* x0,
               double* psi, double* phi, amgt_stats* st);

/* Solves n independent problems, one context each, concurrently: nthreads
 * host threads (0: min(n, 16)) each drive amgt_solve on the next context,
 * and every context issues its work on its own stream -- give each context
 * its own stream, contexts sharing a stream run one after another.  opt
 * applies to all; psi[i] / phi[i] (phi may be NULL) as in amgt_solve, stats
 * (may be NULL) receives n entries.  Each solve is followed by amgt_sync, so
 * a bounded device-side wait that gave up is reported as that problem's
 * status (the cooperative coarse solvers rely on the co-residency that a
 * cooperative launch guarantees its blocks).  The contexts must be non-null
 * and distinct (AMGT_ERR_ARG before any work otherwise).  Returns the first
 * non-OK status of the n solves (all of them run). */
int amgt_solve_batch(amgt_ctx* const* ctxs, int n, const amgt_options* opt, double* const* psi,
                     double* const* phi, amgt_stats* stats, int nthreads);

/* Builds the n contexts' set-up tables (what the first use of a context
 * would build: angular tables, block inverses, transfer and Gauss-Seidel
 * tables, workspaces of the operators' plans) concurrently on nthreads host
 * threads (0: min(n, 16)), each context on its own stream; a batch of many
 * small problems spends most of its set-up in host work and small
 * synchronous copies, which overlap across contexts this way.  The contexts
 * must be non-null and distinct (AMGT_ERR_ARG before any work otherwise).
 * Returns the first non-OK status (all are attempted). */
int amgt_setup_batch(amgt_ctx* const* ctxs, int n, int nthreads);

/* ---- operators of the hot path on device buffers -------------------------- */
/* All buffers are contiguous [Nsdof][Nadof(level)] of element type `dtype`
 * unless stated; they must not alias unless stated. */

/* f = volumetric source + boundary inflow terms on level k (Sec. 2.3, Q). */
int amgt_op_source(amgt_ctx* ctx, int level, int dtype, void* f);
/* psi = L^-1 b: upwind sweep over the cells per sweep direction, one block
 * solve per (cell, patch) (Sec. 3).  Exact on these meshes. */
int amgt_op_sweep(amgt_ctx* ctx, int level, int dtype, const void* b, void* psi);
/* y = L x (Eq. complete, left-hand side with upwind face fluxes).  dtype
 * AMGT_F64_SPLIT: double buffers, L x in double-float arithmetic on the FP32
 * units (hi + lo FP32 parts, error-free sums and products; relative error
 * ~1e-13 of the terms), the form the mixed solve's refinement residuals use
 * with the split-form scatter. */
int amgt_op_apply_L(amgt_ctx* ctx, int level, int dtype, const void* x, void* y);
/* y = S x: Q_[j,q]lm = sum N_li sum_n sigma_{s,n} X X phi (Sec. 4.2), with the
 * level's scatter order.  dtype AMGT_F32_BF16TC: float buffers, contraction
 * in BF16 on tensor cores with FP32 accumulation; AMGT_F64_SPLIT: double
 * buffers, the dense S_f contraction to FP64 accuracy from BF16 tensor-core
 * products (also accepted by amgt_op_apply_A, amgt_op_smooth and
 * amgt_op_vcycle, where every FP64 scatter takes that form; other operators
 * treat it as AMGT_F64). */
int amgt_op_scatter(amgt_ctx* ctx, int level, int dtype, const void* x, void* y);
/* y = (L - S) x. */
int amgt_op_apply_A(amgt_ctx* ctx, int level, int dtype, const void* x, void* y);
/* rc = P^T rf from level k to level k+1 (R = P^T, Sec. 4.1). */
int amgt_op_restrict(amgt_ctx* ctx, int level, int dtype, const void* rf, void* rc);
/* xf += P xc from level k+1 to level k (Galerkin prolongation, Sec. 4.1). */
int amgt_op_prolong(amgt_ctx* ctx, int level, int dtype, const void* xc, void* xf);
/* nu source iterations phi <- L^-1 (S phi + f) on level k (Sec. 4.1);
 * phi is read and overwritten. */
int amgt_op_smooth(amgt_ctx* ctx, int level, int dtype, int nu, const void* f, void* phi);
/* `sweeps` block Gauss-Seidel sweeps on the coarsest level with self-scatter
 * in each block solve (Sec. 4.2); phi is read and overwritten (left as it
 * is, with no launch, for sweeps = 0). */
int amgt_op_coarse_gs(amgt_ctx* ctx, int dtype, int sweeps, const void* f, void* phi);
/* Same as amgt_op_coarse_gs, but allocates nothing: no cudaMalloc, cudaFree or
 * allocating library call.  Meant for callers that cannot let a library
 * allocate device memory while they run -- a process whose device memory is
 * owned by another framework's caching allocator or held under a fixed
 * budget, or a latency-critical loop that cannot afford an allocation's
 * implicit synchronisation.  The paper has no counterpart to this call.
 * Scratch: the coarsest level's cell flux moments (Nsdof x nmom values of
 * dtype) live in one fixed device array of 32 MiB built into the library,
 * present on every GPU that loads it until the process exits.  Larger
 * coarse levels are rejected with AMGT_ERR_ARG.  Its device address is
 * looked up once per device during context set-up, so set-up must be
 * complete before the call (AMGT_ERR_STATE otherwise; any operator or
 * amgt_query_sizes completes it).  Every call, from every context, uses the
 * same array and leaves its contents behind; each call overwrites it before
 * reading, so no clearing is needed, but calls that overlap on the GPU (other
 * streams, other contexts) race on it and must be serialised by the caller.
 * The library's kernel timers (AMGT_TUNE_KERNEL_TIMERS) never time this call
 * (recording them would create CUDA events), and the moment contraction's and
 * the default row Gauss-Seidel's kernels are resolved at set-up, so a first
 * call does not load their code onto the GPU either. */
int amgt_op_coarse_gs_noalloc(amgt_ctx* ctx, int dtype, int sweeps, const void* f, void* phi);
/* phi = LMG(0, f, finest) (Fig. lmg).  dtype AMGT_F32_BF16TC runs the FP32
 * cycle with the BF16 tensor-core scatter. */
int amgt_op_vcycle(amgt_ctx* ctx, int dtype, const void* f, void* phi);
/* phi_s[Nsdof] = sum_{q,d} psi int Psi_[q]d (zeroth flux moment, Sec. 4.2). */
int amgt_op_scalar_flux(amgt_ctx* ctx, int level, int dtype, const void* psi, void* phi);

/* ---- adjoint and detector-response gradients ------------------------------ */
/* adjoint = 1: every operator, sweep, cycle and solve of this context acts
 * with the transposed operator A^T = L^T - S instead of A.  On these meshes
 * L^T is the same DG operator with every direction reversed (Omega -> -Omega
 * in the streaming terms, upwind sides flipped; Q1 integration by parts and
 * symmetric face and angular mass matrices), and S is symmetric, so the
 * context rebuilds its tables with reversed directions.  With the source of
 * an isotropic emission 4 pi * w[c] (amgt_set_source_iso) and vacuum
 * boundaries, amgt_solve then returns lambda = A^-T g for the response
 * R = sum_c w[c] int_cell phi_s dV.  Returns AMGT_OK; rebuilds lazily. */
int amgt_set_adjoint(amgt_ctx* ctx, int adjoint);
/* R = g^T psi with g this context's source vector on the finest level (for
 * a source 4 pi * w: the response above).  psi [Nsdof][Nadof] FP64, a device
 * pointer if device != 0, else host memory; *R on the host. */
int amgt_response(amgt_ctx* ctx, int device, const double* psi, double* R);
/* Gradients of R = g^T psi, A psi = f, from psi and lambda = A^-T g (both
 * [Nsdof][Nadof] FP64 of the finest level; device pointers if device != 0,
 * else host), with A = L - S of this context's problem (Eq. complete,
 * Sec. 4.2):
 *   dsigma_t[c] = -sum_q lambda_cq^T (N (x) M_q) psi_cq          [C]
 *   dsigma_s[c] =  lambda_c^T (N (x) S_f) psi_c                   [C]
 *   dfmom[m][n] =  sum_{c of material m} sigma_s[c] lambda_c^T (N (x) X_n X_n^T)
 *                  psi_c                                              [nmat][N+1]
 * (S_f = X diag(f_n) X^T, X_n the degree-n harmonics moments; sigma_s[c] the
 * cell's n = 0 scatter cross section).  Outputs in the same memory space as
 * the inputs; the call returns after they are written. */
int amgt_response_gradients(amgt_ctx* ctx, int device, const double* psi, const double* lambda,
                            double* dsigma_t, double* dsigma_s, double* dfmom);

#ifdef __cplusplus
}
#endif
#endif /* AMGT_H */
