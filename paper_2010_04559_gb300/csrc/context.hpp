// Library context: problem statement, set-up tables on host and device,
// workspaces.  Internal to the library.
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <memory>
#include <string>
#include <vector>

#include "amgt.h"
#include "kernels.cuh"
#include "setup.hpp"

namespace amgt {

// device allocation owned by the context
struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  DevMem() = default;
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  ~DevMem() {
    if (p) cudaFree(p);
  }
};

template <class T>
struct LevelDevStore {
  T *K0 = nullptr, *B = nullptr, *Kinv = nullptr, *Aax = nullptr, *Ginv = nullptr, *X = nullptr,
    *XFt = nullptr, *Sqq = nullptr, *w = nullptr, *Aw = nullptr, *Sf = nullptr, *tblk = nullptr,
    *TinvT = nullptr, *SLD = nullptr, *Mang = nullptr;
  // several moment shapes: X^T without f, and f of each shape per moment index
  T *Xt = nullptr, *fdeg = nullptr;
};

struct Level {
  AngMesh mesh;
  int Nr = 0, nmom = 1;
  bool dense = false;   // dense S_f contraction cheaper than the moment form
  std::vector<int> pdir, octant, dir_begin, dir_end;
  int ndir = 0;
  int Emax = 0, Jmax = 0;  // direction-blocked Gauss-Seidel table sizes (coarsest level)
  int gs_vec_ok = 0;      // bit 0: float, bit 1: double vector path of the group GS kernel
  // row-pipelined coarse Gauss-Seidel (coarsest level): blocks, rows per block,
  // materials whose block inverses fit in shared memory and the shared bytes,
  // per precision (blocks 0: not available)
  int rows_nb = 0, rows_rpb = 0;
  int rows_dense[2] = {0, 0};  // per precision: dense form M_d x_c (S_f built)
  int rows_nmat_s[2] = {0, 0}, rows_threads[2] = {0, 0}, rows_gbuf[2] = {0, 0};
  size_t rows_smem[2] = {0, 0};
  int* d_rows = nullptr;                      // [ndir][rows_nb][rows_rpb]
  unsigned long long* d_faces = nullptr;      // tagged face words between rows
  size_t faces_bytes = 0;
  int sweep_G = 0;         // patches per block of the 2D row-pipelined sweep (0: level kernel)
  int chunk_f32 = 0, chunk_f64 = 0;  // 2D sweep staging copy size in bytes (0: no row sweep)
  LevelDevStore<double> d64;
  LevelDevStore<float> d32;
  __nv_bfloat16* Sf_bf16 = nullptr;  // dense S_f^T in BF16 for the tensor-core path
  // FP64 scatter in split form: the rows of S_f cut into BF16 digit slices
  __nv_bfloat16* Sf_split = nullptr;  // [nsl][n][n]
  double* Sf_nu = nullptr;            // [n] row scales (powers of two)
  // FP32-accurate scatter on FP16 tensor cores: [S_hi | S_hi | S_lo] rows of
  // S_f scaled by 2^e, and the inverse scale 2^-e
  __half* Sf_tc3 = nullptr;  // [n][3n]
  double tc3_sinv = 0.0;
  // A^xi_q [P][3][a][a] and M_q [P][a][a] as double-float (hi, lo) pairs
  float2 *df_aax = nullptr, *df_mang = nullptr;
  int *d_pdir = nullptr, *d_octant = nullptr, *d_dbeg = nullptr, *d_dend = nullptr;
  // pencil-beam inflow weights [2 dim][nadof] (null without a beam face)
  double* d_beam = nullptr;
  // transfer to the next coarser level
  int *d_parent = nullptr, *d_cbeg = nullptr, *d_cend = nullptr;
  bool children4 = false;  // coarse patch c has the children 4c..4c+3 on this level
  std::vector<int> task_dir, task_q0, task_nq;
  int *d_task_dir = nullptr, *d_task_q0 = nullptr, *d_task_nq = nullptr;
  long long nsdof = 0;
  int nadof() const { return mesh.nadof(); }
};

struct Workspace {
  // per level: r, f, phi, tmp in each precision
  std::vector<void*> r, f, phi, tmp;
};

}  // namespace amgt

struct amgt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err = "no error";

  // ---- problem statement
  int dim = 0;
  int64_t ncell[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  std::vector<double> sigma_t, sigma_s;
  int N = -1;
  // Legendre moment shapes: nf rows f[m][0..N] (row-major), the shape of each
  // cell (empty when nf == 1)
  int nf = 1;
  std::vector<double> ftab;
  std::vector<int> fid;
  std::vector<double> qsrc;
  int bkind[6] = {0, 0, 0, 0, 0, 0};
  double bval[6] = {0, 0, 0, 0, 0, 0};
  double bdir[6][3] = {};    // kind 3: unit beam direction
  double brange[6][4] = {};  // kind 3: u0, u1, v0, v1 on the face's tangential axes
  int basis = 1;
  std::vector<std::vector<uint8_t>> paths;
  int nlevels = 1;
  std::vector<int> Nr;
  int nu_pre = 1, nu_post = 1, coarse_sweeps = 10;
  bool dirty = true;

  // ---- built state
  amgt::Q1 q1;
  amgt::Geom geom{};
  int C = 0, nmat = 0;
  std::vector<int> mat;
  std::vector<double> mat_st, mat_ss;
  std::vector<int> mat_f;  // moment shape of each material
  std::vector<amgt::Level> lv;
  std::vector<amgt::Transfer> tr;
  std::vector<std::unique_ptr<amgt::DevMem>> mem;  // every device allocation
  int *d_mat = nullptr, *d_cells = nullptr, *d_level_off = nullptr, *d_bkind = nullptr,
      *d_fid = nullptr;
  double *d_sigt = nullptr, *d_sigs = nullptr, *d_q = nullptr, *d_bval = nullptr, *d_mu = nullptr,
         *d_mf = nullptr, *d_brange = nullptr, *d_mat_st = nullptr, *d_mat_ss = nullptr;
  int* d_mat_f = nullptr;
  int* d_setup_flag = nullptr;  // set-up kernels' error flag
  float *d_sigt32 = nullptr, *d_sigs32 = nullptr, *d_Nm32 = nullptr;
  int nlev_wave = 0;
  // scratch
  double* d_partials = nullptr;  // [nblk * 64]
  double* d_dots = nullptr;      // [64]
  void** d_ptrs = nullptr;       // device pointer arrays for multi-vector kernels [256]
  int* d_status = nullptr;
  std::vector<std::vector<void*>> ws64, ws32;  // per level: r, f, phi, tmp
  void* d_moments = nullptr;                   // moment scratch [nsdof * nmom_max] (double)
  size_t moments_bytes = 0;
  void* d_bf16 = nullptr;                      // bf16 operand scratch
  size_t bf16_bytes = 0;
  void* d_split = nullptr;                     // split-form slices, products, row scales
  size_t split_bytes = 0;
  void* d_tc3 = nullptr;                       // FP16 operand rows and row scales
  size_t tc3_bytes = 0;
  int f32_scatter = 0;                         // AMGT_TUNE_F32_SCATTER
  int test_sweep_hold = 0;                     // AMGT_TUNE_TEST_SWEEP_HOLD
  int coarse_f64 = 0;                          // AMGT_TUNE_COARSE_F64
  int fp64_scatter = 0;                        // AMGT_TUNE_FP64_SCATTER
  int split_rows = 0;                          // AMGT_TUNE_SPLIT_ROWS
  int sweep_kernel = 0;                        // AMGT_TUNE_SWEEP_KERNEL
  int gs_cluster = 0;
  void* noalloc_moments = nullptr;  // device address of the fixed moment scratch
  bool adjoint = false;  // amgt_set_adjoint: operators of the transposed problem
  // V-cycle replayed from a captured CUDA graph (AMGT_TUNE_GRAPHS): per
  // precision (0 FP32, 1 FP64) and scatter path (1 tensor cores); the graph
  // reads `in` and writes `out`
  struct VGraph {
    cudaGraphExec_t exec = nullptr;
    void* in = nullptr;
    void* out = nullptr;
    long long nlaunch = 0;
  };
  VGraph vgraph[2][2];
  bool use_graphs = false;
  bool capturing = false;  // a V-cycle is being captured on the stream
  double* d_grad = nullptr;  // gradient scratch (moments, outputs)
  size_t grad_bytes = 0;
  int gs_kernel = 0;    // AMGT_TUNE_GS_KERNEL
  unsigned gs_tag = 0;  // sweeps run by the row-pipelined Gauss-Seidel (face-word tags)
  int gs_grid_blocks = 0;  // AMGT_TUNE_GS_GRID_BLOCKS
  int gs_form = 0;         // AMGT_TUNE_GS_FORM
  int gs_cluster_size = 0; // AMGT_TUNE_GS_CLUSTER
  int sweep_group = 0;  // AMGT_TUNE_SWEEP_GROUP
  int sweep_stages = 0; // AMGT_TUNE_SWEEP_STAGES
  // per-kernel device timers (AMGT_TUNE_KERNEL_TIMERS)
  bool ktimers = false;
  struct KtPending {
    int id;
    cudaEvent_t a, b;
    double work;  // algorithmic bytes or flop of the launch
  };
  std::vector<KtPending> kt_pending;
  std::vector<cudaEvent_t> kt_free;
  double kt_ms[AMGT_KT_COUNT] = {};
  long long kt_n[AMGT_KT_COUNT] = {};
  double kt_work[AMGT_KT_COUNT] = {};
  ~amgt_ctx() {
    for (auto& row : vgraph)
      for (auto& v : row)
        if (v.exec) cudaGraphExecDestroy(v.exec);
    for (auto& p : kt_pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : kt_free) cudaEventDestroy(e);
  }
};
