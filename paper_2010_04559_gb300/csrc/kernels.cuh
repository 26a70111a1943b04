// Device kernels of the transport hot path and their launch wrappers.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

namespace amgt {

constexpr int kMaxS = 8;   // spatial nodes per cell (3D Q1)
constexpr int kMaxA = 3;   // angular functions per patch (Lin)

// Geometry and Q1 constants shared by the transport kernels (per launch).
struct Geom {
  int dim, s, a;
  int nx, ny, nz;
  int C;
  long long nsdof;
  int nadof, P;
  double lo[3], h[3];        // box corner and cell widths
  double facemass[3][4][4];  // [axis][own face node][neighbour face node]
  double Nmass[64];          // spatial mass matrix N (s x s)
  float NmassF[64];
  // streaming matrices of the Kronecker form of L's diagonal block:
  // G[axis][negative Omega component][s*s] (see kernels_transport.cu)
  double Gax[3][2][64];
  float GaxF[3][2][64];
};

// Tables of one angular level in precision T.
template <class T>
struct LevelDev {
  const T* K0;     // [P][sa][sa] streaming part of the diagonal block
  const T* B;      // [P][sa][sa] kron(N, M_q)
  const T* Kinv;   // [nmat][P][sa][sa] inverse diagonal blocks
  const T* Aax;    // [P][3][a][a] A^xi_q
  const T* Ginv;   // [nmat][P][sa][sa] Gauss-Seidel block inverses (coarsest)
  const T* X;      // [nadof][nmom]
  const T* XFt;    // [nf][nmom][nadof] diag(f_n) X^T per moment shape
  const T* Sqq;    // [nf][P][a][a] self-scatter blocks X_q F X_q^T per shape
  const T* w;      // [nadof] int Psi
  const T* Mang;   // [P][a][a] angular mass M_q
  const int* pdir; // [P] sweep direction of each patch
  int nmom;
};

struct CellData {
  const int* mat;         // [C] material index
  const int* fid;         // [C] moment shape of the cell (null: one shape)
  const double* sigma_t;  // [C]
  const double* sigma_s;  // [C]
  const float* sigma_t32;
  const float* sigma_s32;
};

struct Schedule {
  const int* cells;      // rotated cell coordinates sorted by wavefront level
  const int* level_off;  // [nlev+1]
  int nlev;
  const int* task_dir;   // [ntask]
  const int* task_q0;
  const int* task_nq;
  int ntask;
};

// Raises a kernel's dynamic shared-memory limit to the device's opt-in
// maximum.  The attribute is process-wide per kernel: one fixed value (not each
// launch's own size) keeps launches from concurrent host threads, sized for
// different problems, from undercutting one another.
template <class K>
inline cudaError_t allow_max_smem(K kern) {
  int dev = 0, mx = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  // the opt-in limit covers static and dynamic shared memory together
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              mx - (int)fa.sharedSizeBytes);
}

// status word written by device-side bounded waits
struct DevStatus {
  int* flag;  // device int, 0 = ok
};

// ---- launch wrappers (all asynchronous on `st`) ---------------------------
// G > 0 and dim == 2: row-pipelined kernel with G patches per block (the
// schedule's tasks must then hold G-patch groups); otherwise the level kernel.
template <class T>
// variant: 0 auto, 1 level-synchronous row kernel, 2 warp-pipelined (2D, Lin);
// err: status word for the bounded waits of the warp-pipelined form;
// test_hold != 0 (tests of the failure path only): in the warp-pipelined form
// the first warp of each block never publishes its progress and every wait
// gives up after 10 ms, so the launch ends with status code 7
// 3D (variant 0 or 2): the grid-wide level form when a cooperative launch fits
// (gbar: two words for its grid barrier; a barrier that waits 2 s records
// status code 8), else the per-task level kernel
void launch_sweep(const Geom& g, const LevelDev<T>& t, const CellData& cd, const Schedule& sc,
                  const T* b, T* psi, int G, int nmat, int chunk_bytes, int nst, int variant,
                  int* err, int test_hold, unsigned* gbar, cudaStream_t st);
template <class T>
void launch_apply_L(const Geom& g, const LevelDev<T>& t, const CellData& cd, T alpha, T beta,
                    const T* x, T* y, cudaStream_t st);
// the same FP64 L x in double-float arithmetic (hi + lo FP32 parts, ~44 bits;
// relative error ~1e-13 of the terms) on the FP32 units; aax [P][3][a][a] and
// mang [P][a][a] are A^xi_q and M_q split into (hi, lo) float pairs
void launch_apply_L_df(const Geom& g, const float2* aax, const float2* mang, const int* pdir,
                       const double* sigma_t, double alpha, double beta, const double* x,
                       double* y, cudaStream_t st);
// C[M][N] = A[M][K] B[K][N] with epilogue (see kernels_gemm.cu)
struct GemmEpi {
  int mode;            // 0 store, 1 cell mix: out = alpha*sig_s*Nmix(acc) + beta*out + add
  double alpha, beta;
  const void* add;     // optional [M][N] same type, may be null
  int s;               // rows per cell
  const double* sig;   // per-cell scale (double) for T=double
  const float* sig32;  // per-cell scale for T=float
  double Nm[64];       // spatial mass matrix N (s x s) for the cell mixing
};
template <class T>
void launch_gemm(int M, int N, int K, const T* A, int lda, const T* B, int ldb, T* C, int ldc,
                 const GemmEpi& epi, cudaStream_t st);
cudaError_t preload_gemm();

// Set-up block inverses on the GPU (kernels_setup.cu), FP64: kind 0
// (K0_q + sigma_t B_q)^-1 and kind 1 (... - sigma_s N (x) S_qq)^-1 per material
// and patch into out[nmat][P][sa][sa]; kind 2 the direction-blocked Gauss-
// Seidel inverses per material and direction, transposed and zero-padded
// into out[nmat][ndir][Emax][Emax].  Matrices up to invert_blocks_max().
int invert_blocks_max();
cudaError_t launch_invert_blocks(const Geom& g, int kind, int nmat, int P, int s, int a,
                                 const double* K0, const double* B, const double* Sqq,
                                 const double* SLD, int ndir, const int* dir_begin,
                                 const int* dir_end, int Jmax, int Emax, const double* mat_st,
                                 const double* mat_ss, const int* mat_f, double* out,
                                 int* singular, cudaStream_t st);

template <class T>
// uniform4: every coarse patch c has the children 4c..4c+3 (a thread per
// coarse patch with its coefficients in registers, 16-byte fine-side access)
void launch_restrict(long long nsdof, int Pc, int a, int nadof_f, int nadof_c, const int* cbeg,
                     const int* cend, const T* blk, const T* rf, T* rc, bool uniform4,
                     cudaStream_t st);
template <class T>
void launch_prolong(long long nsdof, int Pf, int a, int nadof_f, int nadof_c, const int* parent,
                    const T* blk, const T* xc, T* xf, bool uniform4, cudaStream_t st);
template <class T>
void launch_source(const Geom& g, const T* w, const T* Aw, const int* octant,
                   const double* q, const double* bnd_val, const int* bnd_kind,
                   const double* beam, const double* brange, const double* mu,
                   const double* mf, T* f, cudaStream_t st);
template <class T>
void launch_scalar_flux(long long nsdof, int nadof, const T* w, const T* psi, T* phi,
                        cudaStream_t st);
template <class T>
void launch_coarse_gs(const Geom& g, const LevelDev<T>& t, const CellData& cd,
                      const Schedule& sc, int ndir, const int* dir_begin, const int* dir_end,
                      int sweeps, const T* f, T* phi, T* moments, int* status,
                      cudaStream_t st);

// direction-blocked coarse Gauss-Seidel (same iteration, see kernels_gs.cu)
template <class T>
void launch_coarse_gs_block(const Geom& g, const LevelDev<T>& t, const CellData& cd,
                            const Schedule& sc, int ndir, const int* dir_begin,
                            const int* dir_end, int sweeps, const T* f, T* phi, T* moments,
                            const T* TinvT, const T* SLD, int Emax, int Jmax, int nmat,
                            int variant, int vec_ok, int max_level_cells, int grid_blocks,
                            unsigned* gbar, int* err, int* status, cudaStream_t st);

// tensor-core form of the direction-blocked coarse Gauss-Seidel (FP32);
// returns the cluster size used, or < 0 if the shape is not supported
int launch_coarse_gs_tc(const Geom& g, const LevelDev<float>& t, const CellData& cd,
                        const Schedule& sc, int ndir, const int* dir_begin, const int* dir_end,
                        const int* hdir_begin, const int* hdir_end, int sweeps, const float* f,
                        float* phi, float* moments, const float* TinvT, const float* SLD, int Emax,
                        int Jmax, int nmat, int cluster_req, cudaStream_t st);

// row-pipelined form of the direction-blocked coarse Gauss-Seidel (see
// kernels_gs_rows.cu).  plan: returns the number of thread blocks that can be
// resident at once (capped by the number of rows ny*nz; 0 if the shapes are
// not supported) with the materials whose inverses fit in shared memory, the
// threads, the shared bytes per block and the size of the per-cell prefetch
// buffers for the other materials' inverses (0: read from global memory).
// dense: the dense form (M_d x_c from S_f, no flux moments; Sf must then be
// given to the launch and mom is not touched).  launch: returns 0 on a
// successful launch.
template <class T>
int coarse_gs_rows_plan(const Geom& g, int ndir, int nmat, int Jmax, int nmom, bool dense,
                        int* nmat_s, int* threads, size_t* smem, int* gbuf);
// the register form of the FP32 dense-form kernel serves this plan
bool coarse_gs_rows_fast(const Geom& g, int Jmax, int nmat, int nmat_s, int threads);
template <class T>
int launch_coarse_gs_rows(const Geom& g, const LevelDev<T>& t, const CellData& cd, int ndir,
                          const int* dir_begin, const int* dir_end, int sweeps, const T* f,
                          T* phi, T* mom, const T* TinvT, const T* SLD, const T* Sf, int Emax,
                          int Jmax, int nmat, int nmat_s, int gbuf, int threads, size_t smem,
                          const int* rows, int nblocks, int rpb, unsigned long long* faces,
                          unsigned tag0, int* err, cudaStream_t st);

// detector-response gradients (kernels_adjoint.cu), FP64:
// dsigt[c] = -sum_q lam_cq^T kron(N, M_q) psi_cq;
// dsigs[c] = sum_k f_deg(k) (PhiL_c^T N PhiP_c)_kk, dfn[n] += sigma_s[c] * the degree-n part
// (dfn must be zeroed first)
void launch_grad_sigma_t(const Geom& g, const double* Mang, const double* psi, const double* lam,
                         double* dsigt, cudaStream_t st);
// ftab [nf][N+1] moment shapes, fid [C] the cell's shape (null: shape 0);
// dfn [nf][N+1]
void launch_grad_moments(const Geom& g, int nmom, int N, const double* PhiP, const double* PhiL,
                         const double* ftab, const int* fid, const double* sig_s, double* dsigs,
                         double* dfn, cudaStream_t st);

// fixed moment scratch of the allocation-free coarse Gauss-Seidel entry point
size_t noalloc_moment_bytes();
cudaError_t noalloc_moment_address(int device, void** out);

// BLAS-1/2 for GMRES (FP64 or FP32); partials has room for blocks*(nvec)
template <class T>
void launch_multidot(long long n, int nvec, const T* const* V, const T* w, double* partials,
                     int nblk, double* out, cudaStream_t st);
template <class T>
void launch_update_multidot(long long n, int nvec, const T* const* V, const double* h, T* w,
                            int do_dot, double* partials, int nblk, double* out,
                            cudaStream_t st);
template <class T>
void launch_axpby(long long n, double alpha, const T* x, double beta, T* y, cudaStream_t st);
template <class T>
void launch_scale_copy(long long n, double alpha, const T* x, T* y, cudaStream_t st);
template <class Tin, class Tout>
void launch_convert(long long n, const Tin* x, Tout* y, cudaStream_t st);
// Phi[r][k] *= fdeg[fid[r / s]][k] for r < rows (moments scaled by each
// cell's moment shape)
template <class T>
void launch_scale_moments(long long rows, int s, int nmom, const int* fid, const T* fdeg, T* Phi,
                          cudaStream_t st);
template <class T>
void launch_lincomb(long long n, int nvec, const T* const* Z, const double* y, T* x,
                    cudaStream_t st);
int gemv_blocks(long long n);

// process-wide count of kernels launched by the library
void note_launch(int n = 1);
long long launch_count();

// BF16 tensor-core scatter (tcgen05), see kernels_tc.cu
bool tc_available();
// Xb[c*s+l][:] = bf16(alpha * sig[c] * sum_i N[l][i] x[c*s+i][:])
void launch_tc_prep(long long ncell, int s, int n, const float* x, const float* sig,
                    const float* Nm, float alpha, __nv_bfloat16* xb, cudaStream_t st);
// C = A Bt^T (+ beta C + add); returns 0 on a successful launch
int launch_tc_gemm(int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* Bt, float* C,
                   const float* add, float beta, int* err, cudaStream_t st);
// C = rs (A Bt^T) (+ beta C + add) with A, Bt both BF16 (f16 = false) or both
// FP16 (f16 = true); rs [M] per-row scales or null
int launch_tc_gemm_ex(int M, int N, int K, const void* A, const void* Bt, bool f16, float* C,
                      const float* add, float beta, const float* rs, int* err, cudaStream_t st);
// FP32-accurate scatter on FP16 tensor cores (kernels_tc3.cu): rows r = c s + l
// of z = alpha sig[c] (N x_c)[l] scaled per row by a power of two and cut into
// hi + lo FP16 parts, out[r] = [hi | lo | hi] (3n halves), rs[r] = inverse row
// scale times sinv
void launch_tc3_prep(long long ncell, int s, int n, const float* x, const float* sig,
                     const float* Nm, float alpha, float sinv, __half* out, float* rs,
                     cudaStream_t st);
// Bt[n][3n] = [S_hi | S_hi | S_lo] of S scaled by one power of two (largest
// entry in [2^14, 2^15)); *sinv receives the inverse scale (synchronises st)
cudaError_t tc3_split_sf(int n, const double* Sf, unsigned long long* dmax, __half* Bt,
                         double* sinv, cudaStream_t st);

// Error-free splitting of FP64 rows into BF16 digit slices (kernels_split64.cu):
// per row r of z (x itself, or with mix the per-cell rows sig[c] N x of S
// spatial nodes) mu[r] = 2^e > max |z[r]|, and slice i (0 <= i < nsl) holds
// the integer digits d_i with z = mu sum_i d_i 2^(-bits (i+1)) + remainder.
struct NmassArg {
  double v[64];
};
void launch_split_rows(long long rows, int K, int S, bool mix, const double* x,
                       const double* sig, const double* Nm, int nsl, int bits, double* mu,
                       __nv_bfloat16* out, long long slice_stride, cudaStream_t st);
// y[r][c] += sc mu[r] nu[c] P[r][c] for r < M, c < N (row strides N)
void launch_split_flush(long long M, int N, const float* P, const double* mu, const double* nu,
                        double sc, double* y, cudaStream_t st);

}  // namespace amgt
