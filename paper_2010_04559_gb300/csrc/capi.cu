// C ABI of the library: problem statement, set-up, operator entry points, the
// angular multigrid V-cycle (Fig. lmg) and restarted GMRES (FP64 and the mixed
// FP64-refinement / FP32-flexible-GMRES form).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <initializer_list>
#include <map>
#include <tuple>
#include <mutex>
#include <stdexcept>
#include <string>
#include <thread>
#include <type_traits>
#include <utility>

#include "context.hpp"
#include "split_plan.hpp"

using namespace amgt;

namespace {

#define CK(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return e_ == cudaErrorMemoryAllocation ? AMGT_ERR_NOMEM : AMGT_ERR_CUDA;      \
    }                                                                               \
  } while (0)

#define TRY(expr)                   \
  do {                              \
    int rc_ = (expr);               \
    if (rc_ != AMGT_OK) return rc_; \
  } while (0)

int fail(amgt_ctx* ctx, int code, const std::string& msg) {
  ctx->err = msg;
  return code;
}

template <class T>
int dalloc(amgt_ctx* ctx, size_t n, T** out) {
  auto m = std::make_unique<DevMem>();
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(&m->p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, AMGT_ERR_NOMEM,
                "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed");
  }
  m->bytes = n * sizeof(T);
  *out = static_cast<T*>(m->p);
  ctx->mem.push_back(std::move(m));
  return AMGT_OK;
}

template <class Tdev, class Thost>
int upload(amgt_ctx* ctx, const std::vector<Thost>& h, Tdev** out) {
  TRY(dalloc<Tdev>(ctx, h.size(), out));
  if constexpr (std::is_same<Thost, Tdev>::value) {
    CK(cudaMemcpy(*out, h.data(), h.size() * sizeof(Tdev), cudaMemcpyHostToDevice));
  } else {
    // converted in chunks (tables of many materials reach tens of GB)
    const size_t chunk = (size_t)1 << 24;
    std::vector<Tdev> tmp(std::min(chunk, h.size()));
    for (size_t b = 0; b < h.size(); b += chunk) {
      const size_t n = std::min(chunk, h.size() - b);
      for (size_t i = 0; i < n; ++i) tmp[i] = (Tdev)h[b + i];
      CK(cudaMemcpy(*out + b, tmp.data(), n * sizeof(Tdev), cudaMemcpyHostToDevice));
    }
  }
  return AMGT_OK;
}

int nmoments(int N) { return (N + 1) * (N + 1); }

// fn(i) for i in [0, n) on the host's cores (set-up tables: one block inverse
// per (material, patch) -- millions when every cell has its own sigma_t)
template <class F>
void parallel_for(long long n, F fn) {
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 1;
  if (nt > 64) nt = 64;
  if (n < 256 || nt == 1) {
    for (long long i = 0; i < n; ++i) fn(i);
    return;
  }
  std::atomic<long long> next{0};
  std::vector<std::thread> ts;
  for (unsigned t = 0; t < nt; ++t)
    ts.emplace_back([&] {
      for (long long i; (i = next.fetch_add(1)) < n;) fn(i);
    });
  for (auto& t : ts) t.join();
}

// largest number of cells on one wavefront level i + j + k = const
int max_wavefront_cells(const Geom& g) {
  std::vector<int> cnt(g.nx + g.ny + g.nz, 0);
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) cnt[i + j + k]++;
  return *std::max_element(cnt.begin(), cnt.end());
}

// kron(S[s][s], Ang[a][a]) accumulated with factor into out[(s a)^2]
void kron_add(int s, int a, const double* S, const double* Ang, double fac, double* out) {
  const int sa = s * a;
  for (int l = 0; l < s; ++l)
    for (int i = 0; i < s; ++i) {
      const double sv = S[l * s + i] * fac;
      if (sv == 0.0) continue;
      for (int m = 0; m < a; ++m)
        for (int d = 0; d < a; ++d) out[(l * a + m) * sa + i * a + d] += sv * Ang[m * a + d];
    }
}

template <class T>
LevelDev<T> level_view(const Level& L, const LevelDevStore<T>& s) {
  LevelDev<T> v;
  v.K0 = s.K0;
  v.B = s.B;
  v.Kinv = s.Kinv;
  v.Aax = s.Aax;
  v.Ginv = s.Ginv;
  v.X = s.X;
  v.XFt = s.XFt;
  v.Sqq = s.Sqq;
  v.w = s.w;
  v.Mang = s.Mang;
  v.pdir = L.d_pdir;
  v.nmom = L.nmom;
  return v;
}

template <class T>
const LevelDevStore<T>& store(const Level& L);
template <>
const LevelDevStore<double>& store<double>(const Level& L) {
  return L.d64;
}
template <>
const LevelDevStore<float>& store<float>(const Level& L) {
  return L.d32;
}

Geom level_geom(const amgt_ctx* ctx, int k) {
  Geom g = ctx->geom;
  g.nadof = ctx->lv[k].nadof();
  g.P = ctx->lv[k].mesh.P;
  g.a = ctx->lv[k].mesh.a;
  return g;
}

// CUDA events around one launch on the context's stream while the kernel
// timers are on (RAII: the stop event is recorded when the scope ends), with
// the launch's algorithmic work (bytes or flop, per kernel class)
struct KernelTimer {
  amgt_ctx* ctx;
  int id;
  double work;
  cudaEvent_t a = nullptr, b = nullptr;
  static cudaEvent_t take(amgt_ctx* c) {
    if (!c->kt_free.empty()) {
      cudaEvent_t e = c->kt_free.back();
      c->kt_free.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
  // enabled = false: never records (the allocation-free entry point, which
  // must not create events)
  KernelTimer(amgt_ctx* c, int kid, double w = 0.0, bool enabled = true)
      : ctx(c), id(kid), work(w) {
    if (!ctx->ktimers || !enabled) return;
    a = take(ctx);
    b = take(ctx);
    if (!a || !b) {
      if (a) ctx->kt_free.push_back(a);
      if (b) ctx->kt_free.push_back(b);
      a = b = nullptr;
      return;
    }
    cudaEventRecord(a, ctx->stream);
  }
  ~KernelTimer() {
    if (!a) return;
    cudaEventRecord(b, ctx->stream);
    ctx->kt_pending.push_back({id, a, b, work});
  }
};

CellData cell_data(const amgt_ctx* ctx) {
  CellData cd;
  cd.mat = ctx->d_mat;
  cd.fid = ctx->nf > 1 ? ctx->d_fid : nullptr;
  cd.sigma_t = ctx->d_sigt;
  cd.sigma_s = ctx->d_sigs;
  cd.sigma_t32 = ctx->d_sigt32;
  cd.sigma_s32 = ctx->d_sigs32;
  return cd;
}

Schedule schedule(const amgt_ctx* ctx, int k) {
  const Level& L = ctx->lv[k];
  Schedule sc;
  sc.cells = ctx->d_cells;
  sc.level_off = ctx->d_level_off;
  sc.nlev = ctx->nlev_wave;
  sc.task_dir = L.d_task_dir;
  sc.task_q0 = L.d_task_q0;
  sc.task_nq = L.d_task_nq;
  sc.ntask = (int)L.task_dir.size();
  return sc;
}

// ---------------------------------------------------------------- set-up
template <class T>
int upload_level(amgt_ctx* ctx, Level& L, const std::vector<double>& K0,
                 const std::vector<double>& B, const std::vector<double>& Kinv,
                 const std::vector<double>& Ginv, const std::vector<double>& X,
                 const std::vector<double>& XFt, const std::vector<double>& Sqq,
                 const std::vector<double>& tblk, LevelDevStore<T>& s,
                 const std::vector<double>& Xt = {}, const std::vector<double>& fdeg = {}) {
  TRY(upload(ctx, K0, &s.K0));
  TRY(upload(ctx, B, &s.B));
  if (!Kinv.empty()) TRY(upload(ctx, Kinv, &s.Kinv));
  TRY(upload(ctx, L.mesh.A, &s.Aax));
  if (!Ginv.empty()) TRY(upload(ctx, Ginv, &s.Ginv));
  TRY(upload(ctx, X, &s.X));
  TRY(upload(ctx, XFt, &s.XFt));
  TRY(upload(ctx, Sqq, &s.Sqq));
  TRY(upload(ctx, L.mesh.w, &s.w));
  TRY(upload(ctx, L.mesh.Aw, &s.Aw));
  TRY(upload(ctx, L.mesh.M, &s.Mang));
  if (!tblk.empty()) TRY(upload(ctx, tblk, &s.tblk));
  if (!Xt.empty()) TRY(upload(ctx, Xt, &s.Xt));
  if (!fdeg.empty()) TRY(upload(ctx, fdeg, &s.fdeg));
  return AMGT_OK;
}

// A^xi_q and M_q as (hi, lo) float pairs for the double-float L apply
int upload_df_tables(amgt_ctx* ctx, Level& L) {
  auto split = [](const std::vector<double>& v) {
    std::vector<float2> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
      const float h = (float)v[i];
      o[i] = make_float2(h, (float)(v[i] - (double)h));
    }
    return o;
  };
  TRY(upload(ctx, split(L.mesh.A), &L.df_aax));
  TRY(upload(ctx, split(L.mesh.M), &L.df_mang));
  return AMGT_OK;
}

// Block inverses of level Lv on the GPU from its uploaded K0, B and S_qq:
// Kinv = (K0_q + sigma_t B_q)^-1 per material and patch, and on the coarsest
// level Ginv = (K0_q + sigma_t B_q - sigma_s N (x) S_qq)^-1; FP32 copies.
int device_block_inverses(amgt_ctx* ctx, Level& Lv, bool coarsest) {
  const int s = ctx->q1.s, a = Lv.mesh.a, P = Lv.mesh.P, sa = s * a;
  const size_t nblk = (size_t)ctx->nmat * P * sa * sa;
  int* sing = ctx->d_setup_flag;
  if (!sing) {
    TRY(dalloc(ctx, 1, &sing));
    ctx->d_setup_flag = sing;
  }
  CK(cudaMemsetAsync(sing, 0, sizeof(int), ctx->stream));
  for (int kind = 0; kind < (coarsest ? 2 : 1); ++kind) {
    double* out64;
    float* out32;
    TRY(dalloc(ctx, nblk, &out64));
    TRY(dalloc(ctx, nblk, &out32));
    CK(launch_invert_blocks(ctx->geom, kind, ctx->nmat, P, s, a, Lv.d64.K0, Lv.d64.B,
                            Lv.d64.Sqq, nullptr, 0, nullptr, nullptr, 0, 0, ctx->d_mat_st,
                            ctx->d_mat_ss, ctx->d_mat_f, out64, sing, ctx->stream));
    launch_convert<double, float>((long long)nblk, out64, out32, ctx->stream);
    CK(cudaGetLastError());
    if (kind == 0) {
      Lv.d64.Kinv = out64;
      Lv.d32.Kinv = out32;
    } else {
      Lv.d64.Ginv = out64;
      Lv.d32.Ginv = out32;
    }
  }
  int h = 0;
  CK(cudaMemcpyAsync(&h, sing, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h) return fail(ctx, AMGT_ERR_ARG, "singular transport or Gauss-Seidel block");
  return AMGT_OK;
}

// Coarse Gauss-Seidel in direction-blocked form: for each material and sweep
// direction d, T = blockdiag_q(K0_q + sigma_t B_q) - sigma_s N (x) S_dd^{L+D}
// over the entries e = l*J + (q - q_b)*a + m, and its inverse (stored
// transposed); S_dd^{L+D} keeps the scatter blocks S_qp with p <= q.
int build_gs_blocks(amgt_ctx* ctx, Level& Lv, const std::vector<double>& K0,
                    const std::vector<double>& B, const std::vector<double>& X,
                    const std::vector<double>& F) {
  const int s = ctx->q1.s, a = Lv.mesh.a, nm = Lv.nmom, sa = s * a;
  int Jmax = 0;
  for (int d = 0; d < Lv.ndir; ++d) Jmax = std::max(Jmax, (Lv.dir_end[d] - Lv.dir_begin[d]) * a);
  const int Emax = s * Jmax;
  Lv.Jmax = Jmax;
  Lv.Emax = Emax;
  // 16-byte vector loads need every direction's J to be a multiple of 4 floats / 2 doubles
  Lv.gs_vec_ok = 3;
  for (int d = 0; d < Lv.ndir; ++d) {
    const int J = (Lv.dir_end[d] - Lv.dir_begin[d]) * a;
    if (J % 4) Lv.gs_vec_ok &= ~1;
    if (J % 2) Lv.gs_vec_ok &= ~2;
  }
  // the per-patch kernel handles larger directions and very many materials
  if (Emax > 384 || (size_t)ctx->nmat * Lv.ndir * Emax * Emax * sizeof(double) > ((size_t)8 << 30))
    return AMGT_OK;
  std::vector<double> SLD((size_t)Lv.ndir * Jmax * Jmax, 0.0);
  const bool dev_inv = Emax <= invert_blocks_max();
  std::vector<double> TinvT(dev_inv ? 0 : (size_t)ctx->nmat * Lv.ndir * Emax * Emax, 0.0);
  for (int d = 0; d < Lv.ndir; ++d) {
    const int qb = Lv.dir_begin[d], J = (Lv.dir_end[d] - qb) * a, E = s * J;
    double* sl = &SLD[(size_t)d * Jmax * Jmax];
    for (int j = 0; j < J; ++j)
      for (int j2 = 0; j2 < J; ++j2) {
        const int q = j / a, p = j2 / a;
        if (p > q) continue;
        double acc = 0.0;
        const double* xa = &X[(size_t)(qb * a + j) * nm];
        const double* xb = &X[(size_t)(qb * a + j2) * nm];
        for (int kk = 0; kk < nm; ++kk) acc += xa[kk] * F[kk] * xb[kk];
        sl[j * Jmax + j2] = acc;
      }
    if (E == 0 || dev_inv) continue;
    std::atomic<int> singular{0};
    parallel_for(ctx->nmat, [&](long long mi) {
      const int mt = (int)mi;
      std::vector<double> T((size_t)E * E, 0.0), Ti((size_t)E * E);
      for (int l = 0; l < s; ++l)
        for (int j = 0; j < J; ++j) {
          const int e = l * J + j, q = j / a, m = j % a;
          for (int i = 0; i < s; ++i)
            for (int j2 = 0; j2 < J; ++j2) {
              const int e2 = i * J + j2, p = j2 / a, dd = j2 % a;
              double v = 0.0;
              if (p == q) {
                const size_t o = (size_t)(qb + q) * sa * sa + (size_t)(l * a + m) * sa + i * a + dd;
                v += K0[o] + ctx->mat_st[mt] * B[o];
              }
              v -= ctx->mat_ss[mt] * ctx->q1.N[l * s + i] * sl[j * Jmax + j2];
              T[(size_t)e * E + e2] = v;
            }
        }
      if (!invert(E, T.data(), Ti.data())) {
        singular = 1;
        return;
      }
      double* out = &TinvT[((size_t)mt * Lv.ndir + d) * Emax * Emax];
      for (int r = 0; r < E; ++r)
        for (int cc = 0; cc < E; ++cc) out[(size_t)cc * Emax + r] = Ti[(size_t)r * E + cc];
    });
    if (singular) return fail(ctx, AMGT_ERR_ARG, "singular direction-blocked Gauss-Seidel matrix");
  }
  TRY(upload(ctx, SLD, &Lv.d64.SLD));
  TRY(upload(ctx, SLD, &Lv.d32.SLD));
  if (!dev_inv) {
    TRY(upload(ctx, TinvT, &Lv.d64.TinvT));
    TRY(upload(ctx, TinvT, &Lv.d32.TinvT));
    return AMGT_OK;
  }
  // on the GPU: one block per (material, direction)
  const size_t n = (size_t)ctx->nmat * Lv.ndir * Emax * Emax;
  double* t64;
  float* t32;
  TRY(dalloc(ctx, n, &t64));
  TRY(dalloc(ctx, n, &t32));
  int* sing = ctx->d_setup_flag;
  if (!sing) {
    TRY(dalloc(ctx, 1, &sing));
    ctx->d_setup_flag = sing;
  }
  CK(cudaMemsetAsync(sing, 0, sizeof(int), ctx->stream));
  CK(launch_invert_blocks(ctx->geom, 2, ctx->nmat, Lv.mesh.P, s, a, Lv.d64.K0, Lv.d64.B,
                          Lv.d64.Sqq, Lv.d64.SLD, Lv.ndir, Lv.d_dbeg, Lv.d_dend, Jmax, Emax,
                          ctx->d_mat_st, ctx->d_mat_ss, ctx->d_mat_f, t64, sing, ctx->stream));
  launch_convert<double, float>((long long)n, t64, t32, ctx->stream);
  CK(cudaGetLastError());
  int h = 0;
  CK(cudaMemcpyAsync(&h, sing, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h) return fail(ctx, AMGT_ERR_ARG, "singular direction-blocked Gauss-Seidel matrix");
  Lv.d64.TinvT = t64;
  Lv.d32.TinvT = t32;
  return AMGT_OK;
}

// Captured V-cycle graphs refer to the context's buffers and tuning: dropped
// whenever either changes.
void drop_graphs(amgt_ctx* ctx) {
  for (auto& row : ctx->vgraph)
    for (auto& v : row) {
      if (v.exec) cudaGraphExecDestroy(v.exec);
      v = amgt_ctx::VGraph();
    }
}

// Sweep tasks of one level: groups of G patches of one sweep direction (2D:
// the row-pipelined kernel's blocks of ny * G threads; 3D: enough patches per
// block to keep about 256 threads busy on a wavefront level).  Gwant > 0
// forces G (autotuning); else the context's AMGT_TUNE_SWEEP_GROUP or the
// heuristic.  Uploads the task arrays.
int make_sweep_tasks(amgt_ctx* ctx, Level& Lv, const Geom& g, int Gwant) {
  const int dim = g.dim, P = Lv.mesh.P, a = Lv.mesh.a, nadof = Lv.nadof();
  Lv.task_dir.clear();
  Lv.task_q0.clear();
  Lv.task_nq.clear();
  int G;
  if (dim == 2) {
    // prefer >= ~120 blocks
    G = 8;
    while (G > 1 && (g.ny * G > 512 || P / G < 120)) G /= 2;
  } else {
    G = std::max(1, std::min(16, 256 / std::max(1, max_wavefront_cells(g))));
  }
  if (ctx->sweep_group > 0) G = ctx->sweep_group;
  if (Gwant > 0) G = Gwant;
  if (dim == 2 && g.ny * G > 512) G = std::max(1, 512 / g.ny);
  Lv.sweep_G = dim == 2 ? G : 0;
  for (int d = 0; d < Lv.ndir; ++d)
    for (int q0 = Lv.dir_begin[d]; q0 < Lv.dir_end[d]; q0 += G) {
      Lv.task_dir.push_back(d);
      Lv.task_q0.push_back(q0);
      Lv.task_nq.push_back(std::min(G, Lv.dir_end[d] - q0));
    }
  // 16-byte staging copies need 16-byte aligned segment starts and lengths
  // copy chunk of the 2D sweep's staging: 16 bytes when every segment start
  // and length is 16-byte aligned, else 8, else one element
  Lv.chunk_f32 = Lv.chunk_f64 = 0;
  if (dim == 2) {
    for (int bytes : {4, 8}) {
      int best = 0;
      for (int ch : {16, 8}) {
        bool ok = true;
        for (size_t i = 0; i < Lv.task_q0.size() && ok; ++i)
          ok = ((size_t)nadof * bytes) % ch == 0 && ((size_t)Lv.task_q0[i] * a * bytes) % ch == 0 &&
               ((size_t)Lv.task_nq[i] * a * bytes) % ch == 0 && ((size_t)G * a * bytes) % ch == 0;
        if (ok) {
          best = ch;
          break;
        }
      }
      (bytes == 4 ? Lv.chunk_f32 : Lv.chunk_f64) = best > 0 ? best : bytes;
    }
  }
  TRY(upload(ctx, Lv.task_dir, &Lv.d_task_dir));
  TRY(upload(ctx, Lv.task_q0, &Lv.d_task_q0));
  TRY(upload(ctx, Lv.task_nq, &Lv.d_task_nq));
  return AMGT_OK;
}

int ensure_dense(amgt_ctx* ctx, int k);

// Row tables and face-word buffer of the row-pipelined coarse Gauss-Seidel:
// block b owns the rows R = b, b + nb, ... (R = iy + ny*iz) in every
// direction, visited in increasing rotated level jy + jz.
int build_gs_rows(amgt_ctx* ctx) {
  const int k = (int)ctx->lv.size() - 1;
  Level& L = ctx->lv[k];
  L.rows_nb = 0;
  L.rows_dense[0] = L.rows_dense[1] = 0;
  if (!L.d32.TinvT || !L.d64.TinvT || L.ndir == 0 || ctx->geom.dim < 2) return AMGT_OK;
  const Geom g = level_geom(ctx, k);
  // the dense form costs J nadof multiply-adds per node and direction, the
  // moment form J nm (source) + J nm (moment update) + J^2 (S_dd^{L+D});
  // in FP32 the dense form also wins where its register kernel applies
  // (measured: 17.7 against 19.7 ms per 10 sweeps at 96 angular unknowns
  // and 25 moments)
  const bool can = ctx->nf == 1 && ctx->gs_form != 1;
  const bool cheaper = ctx->gs_form == 2 || L.nadof() < 2 * L.nmom + L.Jmax;
  int n32 = 0;
  if (can) {
    TRY(ensure_dense(ctx, k));
    n32 = coarse_gs_rows_plan<float>(g, L.ndir, ctx->nmat, L.Jmax, L.nmom, true,
                                     &L.rows_nmat_s[0], &L.rows_threads[0], &L.rows_smem[0],
                                     &L.rows_gbuf[0]);
    L.rows_dense[0] = cheaper || (n32 > 0 && coarse_gs_rows_fast(g, L.Jmax, ctx->nmat,
                                                                 L.rows_nmat_s[0],
                                                                 L.rows_threads[0]));
    L.rows_dense[1] = cheaper;
  }
  if (!L.rows_dense[0])
    n32 = coarse_gs_rows_plan<float>(g, L.ndir, ctx->nmat, L.Jmax, L.nmom, false,
                                     &L.rows_nmat_s[0], &L.rows_threads[0], &L.rows_smem[0],
                                     &L.rows_gbuf[0]);
  const int n64 = coarse_gs_rows_plan<double>(g, L.ndir, ctx->nmat, L.Jmax, L.nmom,
                                              L.rows_dense[1] != 0, &L.rows_nmat_s[1],
                                              &L.rows_threads[1], &L.rows_smem[1],
                                              &L.rows_gbuf[1]);
  int nb = std::min(n32, n64);
  if (ctx->gs_grid_blocks > 0) nb = std::min(nb, ctx->gs_grid_blocks);
  if (nb <= 0) return AMGT_OK;
  const int nrows = g.ny * g.nz;
  const int rpb = (nrows + nb - 1) / nb;
  std::vector<int> rows((size_t)L.ndir * nb * rpb, -1);
  for (int d = 0; d < L.ndir; ++d) {
    const int n1 = g.dim == 2 ? (d & 1) : ((d >> 1) & 1);
    const int n2 = g.dim == 2 ? 0 : (d & 1);
    for (int b = 0; b < nb; ++b) {
      std::vector<std::pair<int, int>> mine;
      for (int R = b; R < nrows; R += nb) {
        const int iy = R % g.ny, iz = R / g.ny;
        const int jy = n1 ? g.ny - 1 - iy : iy, jz = n2 ? g.nz - 1 - iz : iz;
        mine.emplace_back(jy + jz, R);
      }
      std::sort(mine.begin(), mine.end());
      for (size_t i = 0; i < mine.size(); ++i) rows[((size_t)d * nb + b) * rpb + i] = mine[i].second;
    }
  }
  TRY(upload(ctx, rows, &L.d_rows));
  // two words per value (enough for FP64)
  const size_t words = (size_t)(g.dim - 1) * L.ndir * g.C * (g.s / 2) * L.Jmax * 2;
  TRY(dalloc(ctx, words, &L.d_faces));
  L.faces_bytes = words * sizeof(unsigned long long);
  CK(cudaMemset(L.d_faces, 0, L.faces_bytes));
  ctx->gs_tag = 0;
  L.rows_nb = nb;
  L.rows_rpb = rpb;
  return AMGT_OK;
}

// Pencil-beam inflow tables per beam face (kinds 2 and 3, Sec. 5.4, the
// Dirac boundary data taken in the DG weak form): beam[f][q a + m] =
// S |Omega_b . n| share_q Psi_[q]m(Omega_b) from beam_weights (setup.cpp).  A
// normally incident beam (kind 2) points along the inward normal, an
// octahedron vertex, where four patches take 1/4 each at every level.
// Adjoint contexts hold reversed directions (patch q covers -D_q), so their
// table is built from the forward mesh at -Omega_b.
int build_beam(amgt_ctx* ctx, Level& Lv, int dim) {
  bool any = false;
  for (int f = 0; f < 2 * dim; ++f) any |= ctx->bkind[f] >= 2;
  if (!any) return AMGT_OK;
  const int nadof = Lv.mesh.nadof();
  // on an adjoint context patch q stands for -D_q: the same physical beam is
  // found at -Omega_b among the forward patches
  const double sg = ctx->adjoint ? -1.0 : 1.0;
  std::vector<double> beam((size_t)2 * dim * nadof, 0.0);
  for (int f = 0; f < 2 * dim; ++f) {
    if (ctx->bkind[f] < 2) continue;
    double ob[3] = {0.0, 0.0, 0.0}, fac = ctx->bval[f];
    if (ctx->bkind[f] == 2) {
      ob[f / 2] = (f & 1) ? -1.0 : 1.0;
    } else {
      for (int e = 0; e < 3; ++e) ob[e] = ctx->bdir[f][e];
      fac *= std::fabs(ob[f / 2]);  // |Omega_b . n|
    }
    const double om[3] = {sg * ob[0], sg * ob[1], sg * ob[2]};
    const double total = beam_weights(Lv.mesh, om, fac, &beam[(size_t)f * nadof]);
    if (std::fabs(total - 1.0) > 1e-9)
      return fail(ctx, AMGT_ERR_UNSUPPORTED,
                  "beam direction: the patch shares around it do not sum to 1");
  }
  return upload(ctx, beam, &Lv.d_beam);
}

int build(amgt_ctx* ctx) {
  if (!ctx->dirty) return AMGT_OK;
  drop_graphs(ctx);
  if (ctx->dim == 0) return fail(ctx, AMGT_ERR_STATE, "mesh not set");
  if (ctx->N < 0) return fail(ctx, AMGT_ERR_STATE, "materials not set");
  if (ctx->paths.empty()) return fail(ctx, AMGT_ERR_STATE, "angular mesh not set");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->lv.clear();
  ctx->tr.clear();
  ctx->ws64.clear();
  ctx->ws32.clear();
  ctx->mem.clear();
  ctx->d_moments = nullptr;
  ctx->moments_bytes = 0;
  ctx->d_bf16 = nullptr;
  ctx->bf16_bytes = 0;
  // every scratch buffer went with ctx->mem
  ctx->d_split = nullptr;
  ctx->split_bytes = 0;
  ctx->d_tc3 = nullptr;
  ctx->tc3_bytes = 0;
  ctx->d_grad = nullptr;
  ctx->grad_bytes = 0;
  ctx->d_setup_flag = nullptr;
  ctx->d_fid = nullptr;

  const int dim = ctx->dim;
  double h[3] = {1, 1, 1};
  for (int e = 0; e < dim; ++e) h[e] = (ctx->hi[e] - ctx->lo[e]) / (double)ctx->ncell[e];
  ctx->q1 = build_q1(dim, h);
  const Q1& q1 = ctx->q1;
  const int s = q1.s;
  Geom& g = ctx->geom;
  std::memset(&g, 0, sizeof(g));
  g.dim = dim;
  g.s = s;
  g.nx = (int)ctx->ncell[0];
  g.ny = (int)ctx->ncell[1];
  g.nz = dim == 3 ? (int)ctx->ncell[2] : 1;
  for (int e = 0; e < 3; ++e) {
    g.lo[e] = ctx->lo[e];
    g.h[e] = h[e];
  }
  g.C = g.nx * g.ny * g.nz;
  g.nsdof = (long long)g.C * s;
  const int hs = s / 2;
  for (int xi = 0; xi < dim; ++xi)
    for (int jp = 0; jp < hs; ++jp)
      for (int j = 0; j < hs; ++j) g.facemass[xi][jp][j] = q1.facemass[(xi * hs + jp) * hs + j];
  for (int i = 0; i < s * s; ++i) {
    g.Nmass[i] = q1.N[i];
    g.NmassF[i] = (float)q1.N[i];
  }
  // G_xi for a positive / negative Omega_xi (outflow through the high / low face)
  for (int xi = 0; xi < dim; ++xi)
    for (int sg = 0; sg < 2; ++sg)
      for (int i = 0; i < s * s; ++i) {
        const double fo = sg == 0 ? q1.Fown[(size_t)(2 * xi + 1) * s * s + i]
                                  : -q1.Fown[(size_t)(2 * xi) * s * s + i];
        g.Gax[xi][sg][i] = fo - q1.V[(size_t)xi * s * s + i];
        g.GaxF[xi][sg][i] = (float)g.Gax[xi][sg][i];
      }
  CK(cudaGetLastError());
  const int C = g.C;
  ctx->C = C;

  // materials: distinct (sigma_t, sigma_s, moment shape) triples
  std::map<std::tuple<double, double, int>, int> mm;
  ctx->mat.assign(C, 0);
  ctx->mat_st.clear();
  ctx->mat_ss.clear();
  ctx->mat_f.clear();
  const int nf = ctx->nf;
  for (int c = 0; c < C; ++c) {
    const int sh = nf > 1 ? ctx->fid[c] : 0;
    auto key = std::make_tuple(ctx->sigma_t[c], ctx->sigma_s[c], sh);
    auto it = mm.find(key);
    if (it == mm.end()) {
      it = mm.emplace(key, (int)ctx->mat_st.size()).first;
      ctx->mat_st.push_back(ctx->sigma_t[c]);
      ctx->mat_ss.push_back(ctx->sigma_s[c]);
      ctx->mat_f.push_back(sh);
    }
    ctx->mat[c] = it->second;
  }
  ctx->nmat = (int)ctx->mat_st.size();

  TRY(upload(ctx, ctx->mat_st, &ctx->d_mat_st));
  TRY(upload(ctx, ctx->mat_ss, &ctx->d_mat_ss));
  TRY(upload(ctx, ctx->mat_f, &ctx->d_mat_f));
  // angular hierarchy
  const int L = max_level(ctx->paths);
  const int nl = ctx->nlevels;
  if (nl < 1 || L - nl + 1 < 0)
    return fail(ctx, AMGT_ERR_ARG, "multigrid has more levels than the angular hierarchy");
  ctx->lv.resize(nl);
  const int a = ctx->basis == 0 ? 1 : 3;
  const int sa = s * a;
  for (int k = 0; k < nl; ++k) {
    Level& Lv = ctx->lv[k];
    Lv.mesh = build_mesh(coarsen_paths(ctx->paths, L - k), ctx->basis);
    TRY(build_beam(ctx, Lv, dim));  // from the forward patches
    if (ctx->adjoint) {
      // A^T = the same operator with every direction reversed (Omega -> -Omega
      // in the streaming terms, upwind sides flipped); S is symmetric
      for (double& v : Lv.mesh.A) v = -v;
      for (double& v : Lv.mesh.Aw) v = -v;
      for (auto& pt : Lv.mesh.patch) pt.octant ^= 7;
    }
    Lv.nsdof = g.nsdof;
    const int P = Lv.mesh.P;
    const int nadof = Lv.mesh.nadof();
    Lv.Nr = k < (int)ctx->Nr.size() ? std::min(ctx->Nr[k], ctx->N) : ctx->N;
    Lv.nmom = nmoments(Lv.Nr);
    // dense S_f needs one moment shape for every cell
    Lv.dense = nadof < 2 * Lv.nmom && nf == 1;
    const int nm = Lv.nmom;
    std::vector<double> X = x_table(Lv.mesh, Lv.Nr);
    // f of each shape per moment index (degree n of index k: n^2 <= k < (n+1)^2)
    std::vector<double> Fall((size_t)nf * nm);
    for (int sh = 0; sh < nf; ++sh)
      for (int n = 0; n <= Lv.Nr; ++n)
        for (int o = -n; o <= n; ++o)
          Fall[(size_t)sh * nm + n * n + n + o] = ctx->ftab[(size_t)sh * (ctx->N + 1) + n];
    const std::vector<double> F(Fall.begin(), Fall.begin() + nm);  // shape 0
    std::vector<double> XFt((size_t)nf * nm * nadof);
    for (int sh = 0; sh < nf; ++sh)
      for (int j = 0; j < nadof; ++j)
        for (int kk = 0; kk < nm; ++kk)
          XFt[((size_t)sh * nm + kk) * nadof + j] = Fall[(size_t)sh * nm + kk] * X[(size_t)j * nm + kk];
    std::vector<double> Sqq((size_t)nf * P * a * a, 0.0);
    for (int sh = 0; sh < nf; ++sh)
      for (int q = 0; q < P; ++q)
        for (int m = 0; m < a; ++m)
          for (int d = 0; d < a; ++d) {
            double acc = 0.0;
            for (int kk = 0; kk < nm; ++kk)
              acc += X[(size_t)(q * a + m) * nm + kk] * Fall[(size_t)sh * nm + kk] *
                     X[(size_t)(q * a + d) * nm + kk];
            Sqq[(((size_t)sh * P + q) * a + m) * a + d] = acc;
          }
    std::vector<double> Xt;
    if (nf > 1) {
      Xt.resize((size_t)nm * nadof);
      for (int j = 0; j < nadof; ++j)
        for (int kk = 0; kk < nm; ++kk) Xt[(size_t)kk * nadof + j] = X[(size_t)j * nm + kk];
    }
    // per-patch blocks
    std::vector<double> K0((size_t)P * sa * sa, 0.0), B((size_t)P * sa * sa, 0.0);
    Lv.pdir.resize(P);
    Lv.octant.resize(P);
    for (int q = 0; q < P; ++q) {
      const int o = Lv.mesh.patch[q].octant;
      Lv.octant[q] = o;
      Lv.pdir[q] = dim == 2 ? (o >> 1) : o;
      double* K = &K0[(size_t)q * sa * sa];
      for (int xi = 0; xi < dim; ++xi) {
        const int negb = (o >> (2 - xi)) & 1;
        const double* Ax = &Lv.mesh.A[((size_t)q * 3 + xi) * a * a];
        for (int side = 0; side < 2; ++side) {
          const bool outflow = (side == 1) == (negb == 0);
          if (!outflow) continue;
          const double nsgn = side ? 1.0 : -1.0;
          kron_add(s, a, &q1.Fown[(size_t)(2 * xi + side) * s * s], Ax, nsgn, K);
        }
        kron_add(s, a, &q1.V[(size_t)xi * s * s], Ax, -1.0, K);
      }
      kron_add(s, a, q1.N.data(), &Lv.mesh.M[(size_t)q * a * a], 1.0, &B[(size_t)q * sa * sa]);
    }
    const size_t nblk = (size_t)ctx->nmat * P * sa * sa;
    if (nblk * sizeof(double) > (size_t)48 << 30)
      return fail(ctx, AMGT_ERR_UNSUPPORTED,
                  "too many distinct (sigma_t, sigma_s) pairs for per-material block inverses");
    std::vector<double> Kinv, Ginv;
    std::atomic<int> singular{0};
    // the block inverses are built on the GPU (kernels_setup.cu) unless the
    // blocks are larger than it takes
    const bool dev_inv = sa <= invert_blocks_max();
    if (!dev_inv) Kinv.resize(nblk);
    if (!dev_inv) parallel_for((long long)ctx->nmat * P, [&](long long i) {
      const int mt = (int)(i / P), q = (int)(i % P);
      std::vector<double> blk(sa * sa);
      for (int e = 0; e < sa * sa; ++e)
        blk[e] = K0[(size_t)q * sa * sa + e] + ctx->mat_st[mt] * B[(size_t)q * sa * sa + e];
      if (!invert(sa, blk.data(), &Kinv[((size_t)mt * P + q) * sa * sa])) singular = 1;
    });
    if (singular) return fail(ctx, AMGT_ERR_ARG, "singular transport block (sigma_t <= 0?)");
    if (k == nl - 1 && !dev_inv) {
      Ginv.resize(nblk);
      // kron(N, S_qq) per shape and patch
      std::vector<double> NSq((size_t)nf * P * sa * sa, 0.0);
      for (int sq = 0; sq < nf * P; ++sq)
        kron_add(s, a, q1.N.data(), &Sqq[(size_t)sq * a * a], 1.0, &NSq[(size_t)sq * sa * sa]);
      parallel_for((long long)ctx->nmat * P, [&](long long i) {
        const int mt = (int)(i / P), q = (int)(i % P);
        const double* nsq = &NSq[((size_t)ctx->mat_f[mt] * P + q) * sa * sa];
        std::vector<double> blk(sa * sa);
        for (int e = 0; e < sa * sa; ++e)
          blk[e] = K0[(size_t)q * sa * sa + e] + ctx->mat_st[mt] * B[(size_t)q * sa * sa + e] -
                   ctx->mat_ss[mt] * nsq[e];
        if (!invert(sa, blk.data(), &Ginv[((size_t)mt * P + q) * sa * sa])) singular = 1;
      });
      if (singular) return fail(ctx, AMGT_ERR_ARG, "singular Gauss-Seidel block");
    }
    // directions and sweep tasks
    Lv.ndir = dim == 2 ? 4 : 8;
    Lv.dir_begin.assign(Lv.ndir, 0);
    Lv.dir_end.assign(Lv.ndir, 0);
    for (int d = 0; d < Lv.ndir; ++d) {
      int b = -1, e = -1;
      for (int q = 0; q < P; ++q)
        if (Lv.pdir[q] == d) {
          if (b < 0) b = q;
          e = q + 1;
        }
      if (b < 0) b = e = 0;
      Lv.dir_begin[d] = b;
      Lv.dir_end[d] = e;
    }
    TRY(make_sweep_tasks(ctx, Lv, g, 0));
    TRY(upload(ctx, Lv.pdir, &Lv.d_pdir));
    TRY(upload(ctx, Lv.octant, &Lv.d_octant));
    TRY(upload(ctx, Lv.dir_begin, &Lv.d_dbeg));
    TRY(upload(ctx, Lv.dir_end, &Lv.d_dend));
    const std::vector<double> fdeg = nf > 1 ? Fall : std::vector<double>{};
    TRY(upload_level<double>(ctx, Lv, K0, B, Kinv, Ginv, X, XFt, Sqq, {}, Lv.d64, Xt, fdeg));
    TRY(upload_df_tables(ctx, Lv));
    TRY(upload_level<float>(ctx, Lv, K0, B, Kinv, Ginv, X, XFt, Sqq, {}, Lv.d32, Xt, fdeg));
    if (dev_inv) TRY(device_block_inverses(ctx, Lv, k == nl - 1));
    // the direction-blocked Gauss-Seidel tables assume one moment shape; with
    // several, the per-patch kernel (shape-indexed tables) runs
    if (k == nl - 1 && nf == 1) TRY(build_gs_blocks(ctx, Lv, K0, B, X, F));
  }
  for (int k = 0; k + 1 < nl; ++k) {
    Level& F = ctx->lv[k];
    try {
      ctx->tr.push_back(build_transfer(F.mesh, ctx->lv[k + 1].mesh));
    } catch (const std::exception& ex) {
      return fail(ctx, AMGT_ERR_ARG, ex.what());
    }
    const Transfer& t = ctx->tr.back();
    TRY(upload(ctx, t.parent, &F.d_parent));
    {
      const int Pc = (int)t.child_begin.size();
      bool u4 = Pc > 0 && (int)t.parent.size() == 4 * Pc;
      for (int c = 0; u4 && c < Pc; ++c)
        u4 = t.child_begin[c] == 4 * c && t.child_end[c] == 4 * c + 4;
      F.children4 = u4;
    }
    TRY(upload(ctx, t.child_begin, &F.d_cbeg));
    TRY(upload(ctx, t.child_end, &F.d_cend));
    TRY(upload(ctx, t.blk, &F.d64.tblk));
    TRY(upload(ctx, t.blk, &F.d32.tblk));
  }

  // wavefront schedule in rotated coordinates
  {
    const int nlev = g.nx + g.ny + g.nz - 2;
    std::vector<std::vector<int>> byl(nlev);
    for (int jz = 0; jz < g.nz; ++jz)
      for (int jy = 0; jy < g.ny; ++jy)
        for (int jx = 0; jx < g.nx; ++jx) byl[jx + jy + jz].push_back(jx | (jy << 11) | (jz << 22));
    std::vector<int> cells, off(1, 0);
    for (auto& v : byl) {
      cells.insert(cells.end(), v.begin(), v.end());
      off.push_back((int)cells.size());
    }
    ctx->nlev_wave = nlev;
    TRY(upload(ctx, cells, &ctx->d_cells));
    TRY(upload(ctx, off, &ctx->d_level_off));
  }
  // cell data and source
  TRY(upload(ctx, ctx->mat, &ctx->d_mat));
  if (nf > 1) TRY(upload(ctx, ctx->fid, &ctx->d_fid));
  TRY(upload(ctx, ctx->sigma_t, &ctx->d_sigt));
  TRY(upload(ctx, ctx->sigma_s, &ctx->d_sigs));
  TRY(upload(ctx, ctx->sigma_t, &ctx->d_sigt32));
  TRY(upload(ctx, ctx->sigma_s, &ctx->d_sigs32));
  std::vector<double> q = ctx->qsrc;
  if (q.empty()) q.assign(C, 0.0);
  TRY(upload(ctx, q, &ctx->d_q));
  TRY(upload(ctx, std::vector<int>(ctx->bkind, ctx->bkind + 6), &ctx->d_bkind));
  TRY(upload(ctx, std::vector<double>(ctx->bval, ctx->bval + 6), &ctx->d_bval));
  TRY(upload(ctx, std::vector<double>(&ctx->brange[0][0], &ctx->brange[0][0] + 24),
             &ctx->d_brange));
  TRY(upload(ctx, q1.N, &ctx->d_Nm32));
  TRY(upload(ctx, q1.mu, &ctx->d_mu));
  TRY(upload(ctx, q1.mf, &ctx->d_mf));
  // scratch
  TRY(dalloc(ctx, (size_t)gemv_blocks(1LL << 40) * 64, &ctx->d_partials));
  TRY(dalloc(ctx, 64, &ctx->d_dots));
  TRY(dalloc(ctx, 256, &ctx->d_ptrs));
  TRY(dalloc(ctx, 16, &ctx->d_status));
  CK(cudaMemset(ctx->d_status, 0, 16 * sizeof(int)));
  ctx->ws64.assign(nl, {});
  ctx->ws32.assign(nl, {});
  CK(noalloc_moment_address(ctx->device, &ctx->noalloc_moments));
  // the moment contraction's kernels loaded now, not at a first launch inside
  // the allocation-free entry point (the row Gauss-Seidel kernel is resolved
  // by its occupancy query in build_gs_rows)
  CK(preload_gemm());
  TRY(build_gs_rows(ctx));
  ctx->dirty = false;
  return AMGT_OK;
}

int check_level(amgt_ctx* ctx, int k) {
  TRY(build(ctx));
  if (k < 0 || k >= (int)ctx->lv.size()) return fail(ctx, AMGT_ERR_ARG, "level out of range");
  return AMGT_OK;
}

// workspace vector i (0 r, 1 f, 2 phi, 3 tmp, 4 tmp2) of level k in precision T
template <class T>
int wsvec(amgt_ctx* ctx, int k, int i, T** out) {
  auto& ws = sizeof(T) == 8 ? ctx->ws64 : ctx->ws32;
  auto& v = ws[k];
  if ((int)v.size() <= i) v.resize(i + 1, nullptr);
  if (!v[i]) {
    T* p;
    TRY(dalloc<T>(ctx, (size_t)ctx->lv[k].nsdof * ctx->lv[k].nadof(), &p));
    v[i] = p;
  }
  *out = static_cast<T*>(v[i]);
  return AMGT_OK;
}

int moments_scratch(amgt_ctx* ctx, size_t bytes, void** out) {
  if (ctx->moments_bytes < bytes) {
    double* p;
    TRY(dalloc<double>(ctx, (bytes + 7) / 8, &p));
    ctx->d_moments = p;
    ctx->moments_bytes = bytes;
  }
  *out = ctx->d_moments;
  return AMGT_OK;
}

// dense S_f = X diag(f) X^T on the device (FP64), with FP32 and BF16 copies
int ensure_dense(amgt_ctx* ctx, int k) {
  Level& L = ctx->lv[k];
  if (L.d64.Sf) return AMGT_OK;
  const int n = L.nadof();
  double* Sf;
  float* Sf32;
  TRY(dalloc(ctx, (size_t)n * n, &Sf));
  TRY(dalloc(ctx, (size_t)n * n, &Sf32));
  GemmEpi epi{};
  epi.mode = 0;
  launch_gemm<double>(n, n, L.nmom, L.d64.X, L.nmom, L.d64.XFt, n, Sf, n, epi, ctx->stream);
  launch_convert<double, float>((long long)n * n, Sf, Sf32, ctx->stream);
  CK(cudaGetLastError());
  L.d64.Sf = Sf;
  L.d32.Sf = Sf32;
  return AMGT_OK;
}

int ensure_dense_bf16(amgt_ctx* ctx, int k) {
  Level& L = ctx->lv[k];
  if (L.Sf_bf16) return AMGT_OK;
  TRY(ensure_dense(ctx, k));
  const int n = L.nadof();
  __nv_bfloat16* p;
  TRY(dalloc(ctx, (size_t)n * n, &p));
  // S_f is symmetric, so S_f^T (the K-major B operand) equals S_f
  launch_convert<double, __nv_bfloat16>((long long)n * n, L.d64.Sf, p, ctx->stream);
  CK(cudaGetLastError());
  L.Sf_bf16 = p;
  return AMGT_OK;
}

bool split_applies(amgt_ctx* ctx, int k) {
  const int n = ctx->lv[k].nadof();
  return ctx->nf == 1 && tc_available() && n >= 64 && n % 8 == 0 && split_plan(n).bits > 0 &&
         (ctx->geom.s == 4 || ctx->geom.s == 8);
}

// FP64 scatter contraction in split form on this call?  `refinement`: the
// call computes a refinement residual of the mixed solve.
bool use_split64(amgt_ctx* ctx, bool refinement) {
  if (ctx->fp64_scatter == 1) return false;
  if (ctx->fp64_scatter == 2) return true;
  return refinement;
}

// the rows of S_f (symmetric, so also its columns) as digit slices
int ensure_split(amgt_ctx* ctx, int k, const SplitPlan& sp) {
  Level& L = ctx->lv[k];
  if (L.Sf_split) return AMGT_OK;
  TRY(ensure_dense(ctx, k));
  const int n = L.nadof();
  __nv_bfloat16* sl;
  double* nu;
  TRY(dalloc(ctx, (size_t)sp.nsl * n * n, &sl));
  TRY(dalloc(ctx, (size_t)n, &nu));
  launch_split_rows(n, n, 4, false, L.d64.Sf, nullptr, nullptr, sp.nsl, sp.bits, nu, sl,
                    (long long)n * n, ctx->stream);
  CK(cudaGetLastError());
  L.Sf_split = sl;
  L.Sf_nu = nu;
  return AMGT_OK;
}

// y = alpha S x + beta y + add to FP64 accuracy: the cell-mixed rows
// sig_s N x and the rows of S_f are cut into BF16 digit slices, the slice
// products run as tcgen05 GEMMs whose FP32 sums are exact integers, and each
// group of products is scaled by a power of two and accumulated in FP64.
// Rows are processed in chunks that keep the slices within ~8 GB.
int scatter_split64(amgt_ctx* ctx, int k, const double* x, double* y, double alpha, double beta,
                    const double* add) {
  Level& L = ctx->lv[k];
  const long long M = L.nsdof;
  const int n = L.nadof();
  const int S = ctx->geom.s;
  const SplitPlan sp = split_plan(n);
  TRY(ensure_split(ctx, k, sp));
  const long long total = M * n;
  if (add) {
    launch_axpby<double>(total, 1.0, add, beta, y, ctx->stream);
  } else if (beta == 0.0) {
    CK(cudaMemsetAsync(y, 0, (size_t)total * sizeof(double), ctx->stream));
  } else if (beta != 1.0) {
    launch_scale_copy<double>(total, beta, y, y, ctx->stream);
  }
  const size_t per_row = (size_t)sp.nsl * n * 2 + (size_t)n * 4 + 8;
  long long Mc = (long long)(((size_t)8 << 30) / per_row) / 128 * 128;
  if (ctx->split_rows > 0) Mc = ((long long)ctx->split_rows + 127) / 128 * 128;
  if (Mc < 128) Mc = 128;
  if (Mc > M) Mc = M;
  const size_t slice_bytes = (size_t)sp.nsl * Mc * n * 2;
  const size_t p_off = (slice_bytes + 255) / 256 * 256;
  const size_t mu_off = p_off + ((size_t)Mc * n * 4 + 255) / 256 * 256;
  const size_t need = mu_off + (size_t)Mc * 8;
  if (ctx->split_bytes < need) {
    unsigned char* p;
    TRY(dalloc(ctx, need, &p));
    ctx->d_split = p;
    ctx->split_bytes = need;
  }
  auto* base = static_cast<unsigned char*>(ctx->d_split);
  auto* xs = reinterpret_cast<__nv_bfloat16*>(base);
  auto* P = reinterpret_cast<float*>(base + p_off);
  auto* mu = reinterpret_cast<double*>(base + mu_off);
  for (long long r0 = 0; r0 < M; r0 += Mc) {
    const long long rows = std::min(Mc, M - r0);
    {
      // read x (twice: row maximum, digits), write nsl BF16 digit slices
      KernelTimer kt(ctx, AMGT_KT_SPLIT_AUX, (16.0 + 2.0 * sp.nsl) * rows * n);
      launch_split_rows(rows, n, S, true, x + r0 * n, ctx->d_sigs + r0 / S, ctx->geom.Nmass,
                        sp.nsl, sp.bits, mu, xs, rows * n, ctx->stream);
    }
    for (const SplitPass& pass : sp.passes) {
      for (const SplitGemm& gm : pass.gemms) {
        int rc;
        {
          KernelTimer kt(ctx, AMGT_KT_SPLIT_TC, 2.0 * rows * n * n);
          rc = launch_tc_gemm((int)rows, n, n, xs + (size_t)gm.i * rows * n,
                              L.Sf_split + (size_t)gm.j * n * n, P, nullptr, gm.beta,
                              ctx->d_status, ctx->stream);
        }
        if (rc != 0)
          return fail(ctx, AMGT_ERR_UNSUPPORTED,
                      "tensor-core GEMM launch failed (code " + std::to_string(rc) + ")");
      }
      // read the FP32 products, read and write the FP64 result
      KernelTimer kt(ctx, AMGT_KT_SPLIT_AUX, 20.0 * rows * n);
      launch_split_flush(rows, n, P, mu, L.Sf_nu, alpha * std::ldexp(1.0, -sp.bits * (pass.d + 2)),
                         y + r0 * n, ctx->stream);
    }
  }
  CK(cudaGetLastError());
  return AMGT_OK;
}

// the FP16 three-product form applies on level k (tensor cores present,
// K = Nadof >= 64 and a multiple of 8, Q1 cells)
bool tc3_applies(amgt_ctx* ctx, int k) {
  const int n = ctx->lv[k].nadof();
  return ctx->nf == 1 && tc_available() && n >= 64 && n % 8 == 0 &&
         (ctx->geom.s == 4 || ctx->geom.s == 8);
}

// the rows of S_f cut into FP16 [hi | hi | lo] (kernels_tc3.cu)
int ensure_tc3(amgt_ctx* ctx, int k) {
  Level& L = ctx->lv[k];
  if (L.Sf_tc3) return AMGT_OK;
  TRY(ensure_dense(ctx, k));
  const int n = L.nadof();
  __half* bt;
  TRY(dalloc(ctx, (size_t)n * 3 * n, &bt));
  unsigned long long* mx = reinterpret_cast<unsigned long long*>(ctx->d_status + 8);
  double sinv = 0.0;
  CK(tc3_split_sf(n, L.d64.Sf, mx, bt, &sinv, ctx->stream));
  L.Sf_tc3 = bt;
  L.tc3_sinv = sinv;
  return AMGT_OK;
}

// y = alpha S x + beta y + add in FP32 from FP16 tensor-core products: each
// row of alpha sig_s N x is scaled by a power of two and cut into hi + lo
// FP16 parts, and hi S_hi + lo S_hi + hi S_lo run as one GEMM over the
// concatenated inner dimension 3 Nadof, the epilogue undoing the row scales.
// Rows are processed in passes that keep the FP16 operand within ~4 GB.
int scatter_tc3(amgt_ctx* ctx, int k, const float* x, float* y, double alpha, double beta,
                const float* add) {
  Level& L = ctx->lv[k];
  const long long M = L.nsdof;
  const int n = L.nadof();
  const int S = ctx->geom.s;
  TRY(ensure_tc3(ctx, k));
  long long Mc = (long long)(((size_t)4 << 30) / ((size_t)6 * n)) / 128 * 128;
  if (Mc < 128) Mc = 128;
  if (Mc > M) Mc = M;
  const size_t a_bytes = ((size_t)Mc * 3 * n * 2 + 255) / 256 * 256;
  const size_t need = a_bytes + (size_t)Mc * 4;
  if (ctx->tc3_bytes < need) {
    unsigned char* p;
    TRY(dalloc(ctx, need, &p));
    ctx->d_tc3 = p;
    ctx->tc3_bytes = need;
  }
  auto* base = static_cast<unsigned char*>(ctx->d_tc3);
  auto* A = reinterpret_cast<__half*>(base);
  auto* rs = reinterpret_cast<float*>(base + a_bytes);
  for (long long r0 = 0; r0 < M; r0 += Mc) {
    const long long rows = std::min(Mc, M - r0);
    {
      // read FP32 x, write three FP16 operand parts
      KernelTimer kt(ctx, AMGT_KT_TC3_PREP, 10.0 * rows * n);
      launch_tc3_prep(rows / S, S, n, x + r0 * n, ctx->d_sigs32 + r0 / S, ctx->d_Nm32,
                      (float)alpha, (float)L.tc3_sinv, A, rs, ctx->stream);
    }
    int rc;
    {
      KernelTimer kt(ctx, AMGT_KT_TC3, 2.0 * rows * n * 3.0 * n);
      rc = launch_tc_gemm_ex((int)rows, n, 3 * n, A, L.Sf_tc3, true, y + r0 * n,
                             add ? add + r0 * n : nullptr, (float)beta, rs, ctx->d_status,
                             ctx->stream);
    }
    if (rc != 0)
      return fail(ctx, AMGT_ERR_UNSUPPORTED,
                  "tensor-core GEMM launch failed (code " + std::to_string(rc) + ")");
  }
  CK(cudaGetLastError());
  return AMGT_OK;
}

// y = alpha * S x + beta * y + add  (add may be null).  path: 0 the SIMT
// contraction in T; 1 for T = float the BF16 tensor-core form, for T = double
// the split form (where it applies; else the FP64 SIMT contraction); 2 (T =
// float) the FP32-accurate FP16 three-product form where it applies.
template <class T>
int scatter_impl(amgt_ctx* ctx, int k, int path, const T* x, T* y, double alpha, double beta,
                 const T* add) {
  // several moment shapes: the moment form, each cell's moments scaled by its
  // shape (the dense and tensor-core forms assume one S_f)
  if (ctx->nf > 1) path = 0;
  bool tc = path == 1;
  if constexpr (sizeof(T) == 4) {
    if (path == 2 && tc3_applies(ctx, k)) return scatter_tc3(ctx, k, x, y, alpha, beta, add);
  }
  Level& L = ctx->lv[k];
  const long long M = L.nsdof;
  const int n = L.nadof();
  GemmEpi epi{};
  epi.mode = 1;
  epi.alpha = alpha;
  epi.beta = beta;
  epi.add = add;
  epi.s = ctx->geom.s;
  for (int i = 0; i < epi.s * epi.s; ++i) epi.Nm[i] = ctx->geom.Nmass[i];
  epi.sig = ctx->d_sigs;
  epi.sig32 = ctx->d_sigs32;
  // the tensor-core path needs K = Nadof >= 64 (one K step of the tile) and a
  // multiple of 8 (16-byte TMA rows); other levels take the SIMT contraction
  if (tc && (n < 64 || n % 8 != 0)) tc = false;
  if (tc) {
    if constexpr (sizeof(T) == 4) {
      if (!tc_available()) return fail(ctx, AMGT_ERR_UNSUPPORTED, "tensor-core path unavailable");
      TRY(ensure_dense_bf16(ctx, k));
      size_t need = (size_t)M * n * sizeof(__nv_bfloat16);
      if (ctx->bf16_bytes < need) {
        __nv_bfloat16* p;
        TRY(dalloc(ctx, (size_t)M * n, &p));
        ctx->d_bf16 = p;
        ctx->bf16_bytes = need;
      }
      auto* xb = static_cast<__nv_bfloat16*>(ctx->d_bf16);
      // sigma_s and the spatial mass commute with S: applied while rounding to BF16
      {
        KernelTimer kt(ctx, AMGT_KT_SCATTER_PREP, 6.0 * M * n);
        launch_tc_prep(M / ctx->geom.s, ctx->geom.s, n, x, ctx->d_sigs32, ctx->d_Nm32,
                       (float)alpha, xb, ctx->stream);
      }
      int rc;
      {
        KernelTimer kt(ctx, AMGT_KT_SCATTER_TC, 2.0 * M * n * n);
        rc = launch_tc_gemm((int)M, n, n, xb, L.Sf_bf16, y, add, (float)beta, ctx->d_status,
                            ctx->stream);
      }
      if (rc != 0)
        return fail(ctx, AMGT_ERR_UNSUPPORTED,
                    "tensor-core GEMM launch failed (code " + std::to_string(rc) + ")");
      CK(cudaGetLastError());
      return AMGT_OK;
    } else {
      if (split_applies(ctx, k)) return scatter_split64(ctx, k, x, y, alpha, beta, add);
    }
  }
  if (L.dense) {
    TRY(ensure_dense(ctx, k));
    const T* Sf = store<T>(L).Sf;
    KernelTimer kt(ctx, sizeof(T) == 8 ? AMGT_KT_SCATTER_F64 : AMGT_KT_SCATTER_F32,
                   2.0 * M * n * n);
    launch_gemm<T>((int)M, n, n, x, n, Sf, n, y, n, epi, ctx->stream);
  } else {
    void* mp;
    TRY(moments_scratch(ctx, (size_t)M * L.nmom * sizeof(T), &mp));
    T* Phi = static_cast<T*>(mp);
    GemmEpi e0{};
    e0.mode = 0;
    KernelTimer kt(ctx, sizeof(T) == 8 ? AMGT_KT_SCATTER_F64 : AMGT_KT_SCATTER_F32,
                   4.0 * M * n * L.nmom);
    launch_gemm<T>((int)M, L.nmom, n, x, n, store<T>(L).X, L.nmom, Phi, L.nmom, e0, ctx->stream);
    if (ctx->nf > 1) {
      launch_scale_moments<T>(M, ctx->geom.s, L.nmom, ctx->d_fid, store<T>(L).fdeg, Phi,
                              ctx->stream);
      launch_gemm<T>((int)M, n, L.nmom, Phi, L.nmom, store<T>(L).Xt, n, y, n, epi, ctx->stream);
    } else {
      launch_gemm<T>((int)M, n, L.nmom, Phi, L.nmom, store<T>(L).XFt, n, y, n, epi, ctx->stream);
    }
  }
  CK(cudaGetLastError());
  return AMGT_OK;
}

template <class T>
int sweep_impl(amgt_ctx* ctx, int k, const T* b, T* psi) {
  const Level& L = ctx->lv[k];
  const int chunk = sizeof(T) == 4 ? L.chunk_f32 : L.chunk_f64;
  // read b, write psi
  KernelTimer kt(ctx, AMGT_KT_SWEEP, 2.0 * sizeof(T) * L.nsdof * L.nadof());
  launch_sweep<T>(level_geom(ctx, k), level_view<T>(L, store<T>(L)), cell_data(ctx),
                  schedule(ctx, k), b, psi, L.sweep_G, ctx->nmat, chunk, ctx->sweep_stages,
                  ctx->sweep_kernel, ctx->d_status, ctx->test_sweep_hold,
                  reinterpret_cast<unsigned*>(ctx->d_status + 12), ctx->stream);
  CK(cudaGetLastError());
  return AMGT_OK;
}

template <class T>
int applyL_impl(amgt_ctx* ctx, int k, T alpha, T beta, const T* x, T* y) {
  const Level& L = ctx->lv[k];
  // read x, write y (and read y when it accumulates)
  KernelTimer kt(ctx, AMGT_KT_APPLY_L,
                 (beta != T(0) ? 3.0 : 2.0) * sizeof(T) * L.nsdof * L.nadof());
  launch_apply_L<T>(level_geom(ctx, k), level_view<T>(L, store<T>(L)), cell_data(ctx), alpha,
                    beta, x, y, ctx->stream);
  CK(cudaGetLastError());
  return AMGT_OK;
}

// y = alpha L x + beta y in FP64 from double-float arithmetic on the FP32
// units (relative error ~1e-13 of the terms; kernels_transport.cu)
int applyL_df(amgt_ctx* ctx, int k, double alpha, double beta, const double* x, double* y) {
  const Level& L = ctx->lv[k];
  KernelTimer kt(ctx, AMGT_KT_APPLY_L, (beta != 0.0 ? 3.0 : 2.0) * 8.0 * L.nsdof * L.nadof());
  launch_apply_L_df(level_geom(ctx, k), L.df_aax, L.df_mang, L.d_pdir, ctx->d_sigt, alpha, beta, x,
                    y, ctx->stream);
  CK(cudaGetLastError());
  return AMGT_OK;
}

// y = (L - S) x
template <class T>
int applyA_impl(amgt_ctx* ctx, int k, int path, const T* x, T* y) {
  TRY(scatter_impl<T>(ctx, k, path, x, y, -1.0, 0.0, nullptr));
  return applyL_impl<T>(ctx, k, T(1), T(1), x, y);
}

template <class T>
int source_impl(amgt_ctx* ctx, int k, T* f) {
  const Level& L = ctx->lv[k];
  launch_source<T>(level_geom(ctx, k), store<T>(L).w, store<T>(L).Aw, L.d_octant, ctx->d_q,
                   ctx->d_bval, ctx->d_bkind, L.d_beam, ctx->d_brange, ctx->d_mu, ctx->d_mf, f,
                   ctx->stream);
  CK(cudaGetLastError());
  return AMGT_OK;
}

template <class T>
int restrict_impl(amgt_ctx* ctx, int k, const T* rf, T* rc) {
  const Level& F = ctx->lv[k];
  const Level& Cc = ctx->lv[k + 1];
  launch_restrict<T>(F.nsdof, Cc.mesh.P, F.mesh.a, F.nadof(), Cc.nadof(), F.d_cbeg, F.d_cend,
                     store<T>(F).tblk, rf, rc, F.children4, ctx->stream);
  CK(cudaGetLastError());
  return AMGT_OK;
}

template <class T>
int prolong_impl(amgt_ctx* ctx, int k, const T* xc, T* xf) {
  const Level& F = ctx->lv[k];
  const Level& Cc = ctx->lv[k + 1];
  launch_prolong<T>(F.nsdof, F.mesh.P, F.mesh.a, F.nadof(), Cc.nadof(), F.d_parent,
                    store<T>(F).tblk, xc, xf, F.children4, ctx->stream);
  CK(cudaGetLastError());
  return AMGT_OK;
}

// nu steps of phi <- L^-1 (S phi + f); `zero` = phi is known to be zero
template <class T>
int smooth_impl(amgt_ctx* ctx, int k, bool tc, int nu, const T* f, T* phi, bool zero) {
  T* tmp;
  TRY(wsvec<T>(ctx, k, 3, &tmp));
  for (int it = 0; it < nu; ++it) {
    if (zero && it == 0) {
      TRY(sweep_impl<T>(ctx, k, f, phi));
      continue;
    }
    TRY(scatter_impl<T>(ctx, k, tc, phi, tmp, 1.0, 0.0, f));
    TRY(sweep_impl<T>(ctx, k, tmp, phi));
  }
  return AMGT_OK;
}

template <class T>
int coarse_gs_run(amgt_ctx* ctx, int sweeps, const T* f, T* phi, T* mom, bool timed = true);

template <class T>
int coarse_gs_impl(amgt_ctx* ctx, int sweeps, const T* f, T* phi) {
  const Level& L = ctx->lv.back();
  void* mp;
  TRY(moments_scratch(ctx, (size_t)L.nsdof * L.nmom * sizeof(T), &mp));
  return coarse_gs_run<T>(ctx, sweeps, f, phi, static_cast<T*>(mp));
}

// Same operator with the moments in the library's fixed device array; no
// allocation of any kind.
template <class T>
int coarse_gs_noalloc_impl(amgt_ctx* ctx, int sweeps, const T* f, T* phi) {
  const Level& L = ctx->lv.back();
  const size_t need = (size_t)L.nsdof * L.nmom * sizeof(T);
  if (need > noalloc_moment_bytes())
    return fail(ctx, AMGT_ERR_ARG,
                "coarse level needs " + std::to_string(need) + " bytes of moment scratch; the "
                "allocation-free entry point holds at most " +
                    std::to_string(noalloc_moment_bytes()) + " bytes");
  if (!ctx->noalloc_moments) return fail(ctx, AMGT_ERR_STATE, "fixed scratch not set up");
  return coarse_gs_run<T>(ctx, sweeps, f, phi, static_cast<T*>(ctx->noalloc_moments), false);
}

template <class T>
int coarse_gs_run(amgt_ctx* ctx, int sweeps, const T* f, T* phi, T* mom, bool timed) {
  if (sweeps == 0) return AMGT_OK;  // no sweep: phi is left as it is
  const int k = (int)ctx->lv.size() - 1;
  const Level& L = ctx->lv[k];
  const bool rows = store<T>(L).TinvT && (ctx->gs_kernel == 0 || ctx->gs_kernel == 6) &&
                    L.rows_nb > 0;
  const bool dense = rows && L.rows_dense[sizeof(T) == 4 ? 0 : 1];
  auto moments = [&]() {
    GemmEpi e0{};
    e0.mode = 0;
    launch_gemm<T>((int)L.nsdof, L.nmom, L.nadof(), phi, L.nadof(), store<T>(L).X, L.nmom, mom,
                   L.nmom, e0, ctx->stream);
  };
  if (!dense) moments();
  // sequential per-patch form of the block solves, per (cell, patch, sweep):
  // moment source s a nm, self-scatter s a a, mass mixing s a s, block solve
  // (s a)^2, moment update s nm a multiply-adds (dense form: the source
  // s a nadof, no self-scatter or moment update)
  const double sa = (double)ctx->geom.s * L.mesh.a;
  const double gs_fma = (double)L.nsdof / ctx->geom.s * L.mesh.P * sweeps *
                        ((dense ? sa * L.nadof() : 2.0 * sa * L.nmom + sa * L.mesh.a) +
                         sa * ctx->geom.s + sa * sa);
  KernelTimer kt(ctx, AMGT_KT_COARSE_GS, 2.0 * gs_fma, timed);
  // row-pipelined kernel: the default where available
  if (store<T>(L).TinvT && (ctx->gs_kernel == 0 || ctx->gs_kernel == 6)) {
    const int pi = sizeof(T) == 4 ? 0 : 1;
    if (rows) {
      // restart the face-word tags: before wrap-around, and inside a captured
      // graph (every replay then starts from cleared words and tag 0)
      if (ctx->gs_tag > 0xf0000000u || ctx->capturing) {
        CK(cudaMemsetAsync(L.d_faces, 0, L.faces_bytes, ctx->stream));
        ctx->gs_tag = 0;
      }
      if (launch_coarse_gs_rows<T>(level_geom(ctx, k), level_view<T>(L, store<T>(L)),
                                   cell_data(ctx), L.ndir, L.d_dbeg, L.d_dend, sweeps, f, phi,
                                   mom, store<T>(L).TinvT, store<T>(L).SLD,
                                   dense ? store<T>(L).Sf : nullptr, L.Emax, L.Jmax,
                                   ctx->nmat, L.rows_nmat_s[pi], L.rows_gbuf[pi],
                                   L.rows_threads[pi], L.rows_smem[pi], L.d_rows,
                                   L.rows_nb, L.rows_rpb, L.d_faces, ctx->gs_tag,
                                   ctx->d_status, ctx->stream) == 0) {
        if (!ctx->capturing) ctx->gs_tag += (unsigned)sweeps;
        ctx->gs_cluster = 600;
        return AMGT_OK;
      }
    }
    if (ctx->gs_kernel == 6)
      return fail(ctx, AMGT_ERR_ARG, "row-pipelined Gauss-Seidel not available for this problem");
  }
  if (dense) moments();  // the launch above failed: the other kernels keep moments
  int cl = 0;
  if constexpr (sizeof(T) == 4) {
    if (store<T>(L).TinvT && ctx->gs_kernel == 5) {
      cl = launch_coarse_gs_tc(level_geom(ctx, k), level_view<T>(L, store<T>(L)), cell_data(ctx),
                               schedule(ctx, k), L.ndir, L.d_dbeg, L.d_dend, L.dir_begin.data(),
                               L.dir_end.data(), sweeps, f, phi, mom, store<T>(L).TinvT,
                               store<T>(L).SLD, L.Emax, L.Jmax, ctx->nmat, ctx->gs_cluster_size,
                               ctx->stream);
      if (cl > 0) {
        ctx->gs_cluster = 300 + cl;
        CK(cudaGetLastError());
        return AMGT_OK;
      }
      cl = 0;
    }
  }
  if (store<T>(L).TinvT && ctx->gs_kernel != 1) {
    launch_coarse_gs_block<T>(level_geom(ctx, k), level_view<T>(L, store<T>(L)), cell_data(ctx),
                              schedule(ctx, k), L.ndir, L.d_dbeg, L.d_dend, sweeps, f, phi, mom,
                              store<T>(L).TinvT, store<T>(L).SLD, L.Emax, L.Jmax, ctx->nmat,
                              ctx->gs_kernel, L.gs_vec_ok, max_wavefront_cells(ctx->geom),
                              ctx->gs_cluster_size > 0 ? -ctx->gs_cluster_size : ctx->gs_grid_blocks,
                              reinterpret_cast<unsigned*>(ctx->d_status + 4),
                              ctx->d_status, &cl, ctx->stream);
  } else {
    launch_coarse_gs<T>(level_geom(ctx, k), level_view<T>(L, store<T>(L)), cell_data(ctx),
                        schedule(ctx, k), L.ndir, L.d_dbeg, L.d_dend, sweeps, f, phi, mom, &cl,
                        ctx->stream);
  }
  if (cl == 0) return fail(ctx, AMGT_ERR_CUDA, "coarse Gauss-Seidel cluster launch failed");
  ctx->gs_cluster = cl;
  CK(cudaGetLastError());
  return AMGT_OK;
}

// phi = LMG(0, f, k): phi is overwritten
template <class T>
int vcycle_impl(amgt_ctx* ctx, int k, bool tc, const T* f, T* phi) {
  const Level& L = ctx->lv[k];
  const size_t bytes = (size_t)L.nsdof * L.nadof() * sizeof(T);
  if (k == (int)ctx->lv.size() - 1) {
    if constexpr (sizeof(T) == 4) {
      if (ctx->coarse_f64) {
        // the coarsest solve in FP64 inside the FP32 cycle
        const long long n = L.nsdof * L.nadof();
        double *f64, *phi64;
        TRY(wsvec<double>(ctx, k, 1, &f64));
        TRY(wsvec<double>(ctx, k, 2, &phi64));
        launch_convert<float, double>(n, f, f64, ctx->stream);
        CK(cudaMemsetAsync(phi64, 0, (size_t)n * sizeof(double), ctx->stream));
        TRY(coarse_gs_impl<double>(ctx, ctx->coarse_sweeps, f64, phi64));
        launch_convert<double, float>(n, phi64, phi, ctx->stream);
        CK(cudaGetLastError());
        return AMGT_OK;
      }
    }
    CK(cudaMemsetAsync(phi, 0, bytes, ctx->stream));
    return coarse_gs_impl<T>(ctx, ctx->coarse_sweeps, f, phi);
  }
  TRY(smooth_impl<T>(ctx, k, tc, ctx->nu_pre, f, phi, true));
  if (ctx->nu_pre == 0) CK(cudaMemsetAsync(phi, 0, bytes, ctx->stream));
  T *r, *fc, *phic;
  TRY(wsvec<T>(ctx, k, 0, &r));
  TRY(wsvec<T>(ctx, k + 1, 1, &fc));
  TRY(wsvec<T>(ctx, k + 1, 2, &phic));
  if (ctx->nu_pre >= 1) {
    // the last pre-smoothing sweep solved L phi = t exactly (the sweep
    // inverts L): t = f after one sweep from zero, else S phi_prev + f in
    // workspace 3; so r = f - (L - S) phi = S phi + f - t, with no L apply
    if (ctx->nu_pre == 1) {
      TRY(scatter_impl<T>(ctx, k, tc, phi, r, 1.0, 0.0, nullptr));
    } else {
      T* t;
      TRY(wsvec<T>(ctx, k, 3, &t));
      TRY(scatter_impl<T>(ctx, k, tc, phi, r, 1.0, 0.0, f));
      launch_axpby<T>(L.nsdof * L.nadof(), -1.0, t, 1.0, r, ctx->stream);
      CK(cudaGetLastError());
    }
  } else {
    // r = f - (L - S) phi = (S phi + f) - L phi
    TRY(scatter_impl<T>(ctx, k, tc, phi, r, 1.0, 0.0, f));
    TRY(applyL_impl<T>(ctx, k, T(-1), T(1), phi, r));
  }
  TRY(restrict_impl<T>(ctx, k, r, fc));
  TRY(vcycle_impl<T>(ctx, k + 1, tc, fc, phic));
  TRY(prolong_impl<T>(ctx, k, phic, phi));
  TRY(smooth_impl<T>(ctx, k, tc, ctx->nu_post, f, phi, false));
  return AMGT_OK;
}

// phi = LMG(0, f) on the finest level through a captured CUDA graph: the
// first call runs the cycle directly (every lazy allocation happens there)
// and then captures it reading a fixed input buffer and writing a fixed
// output buffer; later calls copy f in, replay, and copy phi out.
template <class T>
int vcycle_graph(amgt_ctx* ctx, bool tc, const T* f, T* phi) {
  const Level& L0 = ctx->lv[0];
  const size_t bytes = (size_t)L0.nsdof * L0.nadof() * sizeof(T);
  amgt_ctx::VGraph& G = ctx->vgraph[sizeof(T) == 8 ? 1 : 0][tc ? 1 : 0];
  if (!G.exec) {
    TRY(vcycle_impl<T>(ctx, 0, tc, f, phi));
    if (!G.in) {
      T *in, *out;
      TRY(dalloc<T>(ctx, (size_t)L0.nsdof * L0.nadof(), &in));
      TRY(dalloc<T>(ctx, (size_t)L0.nsdof * L0.nadof(), &out));
      G.in = in;
      G.out = out;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    const long long n0 = launch_count();
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = true;
    const int rc = vcycle_impl<T>(ctx, 0, tc, static_cast<const T*>(G.in), static_cast<T*>(G.out));
    ctx->capturing = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (rc != AMGT_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, AMGT_ERR_CUDA, std::string("V-cycle capture: ") + cudaGetErrorString(e));
    }
    const cudaError_t ei = cudaGraphInstantiate(&G.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      G.exec = nullptr;
      cudaGetLastError();
      return fail(ctx, AMGT_ERR_CUDA, std::string("V-cycle graph: ") + cudaGetErrorString(ei));
    }
    G.nlaunch = launch_count() - n0;
    return AMGT_OK;
  }
  CK(cudaMemcpyAsync(G.in, f, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaGraphLaunch(G.exec, ctx->stream));
  CK(cudaMemcpyAsync(phi, G.out, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  note_launch((int)G.nlaunch);
  return AMGT_OK;
}

template <class T>
int scalar_flux_impl(amgt_ctx* ctx, int k, const T* psi, T* phi) {
  const Level& L = ctx->lv[k];
  launch_scalar_flux<T>(L.nsdof, L.nadof(), store<T>(L).w, psi, phi, ctx->stream);
  CK(cudaGetLastError());
  return AMGT_OK;
}

// ------------------------------------------------------------------ GMRES
struct KrylovResult {
  int its = 0;
  int cycles = 0;
  double relres = 0.0;
  int status = AMGT_OK;
};

template <class T>
int dev_dots(amgt_ctx* ctx, int nvec, double* host) {
  CK(cudaMemcpyAsync(host, ctx->d_dots, sizeof(double) * nvec, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return AMGT_OK;
}

template <class T>
int norm2(amgt_ctx* ctx, const T* x, long long n, double* out) {
  const int nblk = gemv_blocks(n);
  void** slot = ctx->d_ptrs + 200;  // kept apart from the Krylov pointer tables
  CK(cudaMemcpyAsync(slot, &x, sizeof(void*), cudaMemcpyHostToDevice, ctx->stream));
  launch_multidot<T>(n, 1, reinterpret_cast<const T* const*>(slot), x, ctx->d_partials,
                     nblk, ctx->d_dots, ctx->stream);
  CK(cudaGetLastError());
  double v;
  TRY(dev_dots<T>(ctx, 1, &v));
  *out = std::sqrt(std::max(v, 0.0));
  return AMGT_OK;
}

// Right-preconditioned GMRES(m), CGS2, Givens rotations, storing the
// preconditioned directions (flexible form).  x holds the initial guess
// (x_zero: known zero) and receives the solution.
template <class T, class OpA, class OpM>
int gmres(amgt_ctx* ctx, int k, OpA apply_A, OpM apply_M, const T* b, T* x, bool x_zero,
          double tol, int m, int maxit, KrylovResult& res, amgt_stats* st, double bnorm_in,
          int hist_base) {
  const long long n = ctx->lv[k].nsdof * ctx->lv[k].nadof();
  const size_t bytes = (size_t)n * sizeof(T);
  m = std::max(1, std::min(m, 30));
  std::vector<T*> V(m + 1), Z(m);
  // Krylov storage is kept in the workspace slots 8.. of level k
  for (int i = 0; i <= m; ++i) TRY(wsvec<T>(ctx, k, 8 + i, &V[i]));
  for (int i = 0; i < m; ++i) TRY(wsvec<T>(ctx, k, 8 + m + 1 + i, &Z[i]));
  T** dV = reinterpret_cast<T**>(ctx->d_ptrs);
  T** dZ = dV + 64;
  CK(cudaMemcpyAsync(dV, V.data(), sizeof(T*) * (m + 1), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(dZ, Z.data(), sizeof(T*) * m, cudaMemcpyHostToDevice, ctx->stream));
  const int nblk = gemv_blocks(n);
  double bnorm = bnorm_in;
  if (bnorm < 0) TRY(norm2<T>(ctx, b, n, &bnorm));
  res = KrylovResult();
  if (bnorm == 0.0) {
    CK(cudaMemsetAsync(x, 0, bytes, ctx->stream));
    return AMGT_OK;
  }
  if (!std::isfinite(bnorm)) return fail(ctx, AMGT_ERR_NAN, "right-hand side is not finite");
  std::vector<double> H((m + 1) * m), cs(m), sn(m), gv(m + 1), h1(m + 1), h2(m + 1), y(m);
  T* r = V[0];
  while (true) {
    if (x_zero) {
      CK(cudaMemcpyAsync(r, b, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
      TRY(apply_A(x, r));
      launch_axpby<T>(n, 1.0, b, -1.0, r, ctx->stream);  // r = b - A x
    }
    double beta;
    TRY(norm2<T>(ctx, r, n, &beta));
    if (!std::isfinite(beta)) return fail(ctx, AMGT_ERR_NAN, "residual is not finite");
    res.relres = beta / bnorm;
    if (res.relres < tol || res.its >= maxit) break;
    launch_scale_copy<T>(n, 1.0 / beta, r, V[0], ctx->stream);
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      TRY(apply_M(V[j], Z[j]));
      T* w = V[j + 1];
      TRY(apply_A(Z[j], w));
      launch_multidot<T>(n, j + 1, dV, w, ctx->d_partials, nblk, ctx->d_dots, ctx->stream);
      CK(cudaGetLastError());
      TRY(dev_dots<T>(ctx, j + 1, h1.data()));
      CK(cudaMemcpyAsync(ctx->d_dots + 32, h1.data(), sizeof(double) * (j + 1),
                         cudaMemcpyHostToDevice, ctx->stream));
      launch_update_multidot<T>(n, j + 1, dV, ctx->d_dots + 32, w, 1, ctx->d_partials, nblk,
                                ctx->d_dots, ctx->stream);
      CK(cudaGetLastError());
      TRY(dev_dots<T>(ctx, j + 1, h2.data()));
      CK(cudaMemcpyAsync(ctx->d_dots + 32, h2.data(), sizeof(double) * (j + 1),
                         cudaMemcpyHostToDevice, ctx->stream));
      launch_update_multidot<T>(n, j + 1, dV, ctx->d_dots + 32, w, 2, ctx->d_partials, nblk,
                                ctx->d_dots, ctx->stream);
      CK(cudaGetLastError());
      double nrm2;
      TRY(dev_dots<T>(ctx, 1, &nrm2));
      const double hn = std::sqrt(std::max(nrm2, 0.0));
      if (!std::isfinite(hn)) return fail(ctx, AMGT_ERR_NAN, "Arnoldi vector is not finite");
      for (int i = 0; i <= j; ++i) H[i * m + j] = h1[i] + h2[i];
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
      }
      const double den = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
      cs[j] = den > 0 ? H[j * m + j] / den : 1.0;
      sn[j] = den > 0 ? H[(j + 1) * m + j] / den : 0.0;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      res.its++;
      jdone = j + 1;
      const double est = std::fabs(gv[j + 1]) / bnorm;
      if (st && hist_base + res.its - 1 < AMGT_MAX_HIST) {
        st->hist[hist_base + res.its - 1] = est;
        st->nhist = hist_base + res.its;
      }
      if (est < tol || res.its >= maxit || hn == 0.0) break;
      launch_scale_copy<T>(n, 1.0 / hn, w, w, ctx->stream);
    }
    for (int i = jdone - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int j2 = i + 1; j2 < jdone; ++j2) acc -= H[i * m + j2] * y[j2];
      if (H[i * m + i] == 0.0) return fail(ctx, AMGT_ERR_BREAKDOWN, "singular Hessenberg");
      y[i] = acc / H[i * m + i];
    }
    if (x_zero) CK(cudaMemsetAsync(x, 0, bytes, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_dots + 32, y.data(), sizeof(double) * jdone,
                       cudaMemcpyHostToDevice, ctx->stream));
    launch_lincomb<T>(n, jdone, reinterpret_cast<const T* const*>(dZ), ctx->d_dots + 32, x,
                      ctx->stream);
    CK(cudaGetLastError());
    x_zero = false;
    res.cycles++;
  }
  return AMGT_OK;
}

// inner products <vecs[i], w>, i < vecs.size() <= 8, in FP64, on the host
template <class T>
int dots_with(amgt_ctx* ctx, long long n, std::initializer_list<const T*> vecs, const T* w,
              double* out) {
  const int nv = (int)vecs.size();
  const T* arr[8];
  int i = 0;
  for (const T* v : vecs) arr[i++] = v;
  void** slot = ctx->d_ptrs + 200;
  CK(cudaMemcpyAsync(slot, arr, sizeof(void*) * nv, cudaMemcpyHostToDevice, ctx->stream));
  launch_multidot<T>(n, nv, reinterpret_cast<const T* const*>(slot), w, ctx->d_partials,
                     gemv_blocks(n), ctx->d_dots, ctx->stream);
  CK(cudaGetLastError());
  return dev_dots<T>(ctx, nv, out);
}

// Right-preconditioned BiCGStab (Sec. 3): shadow residual = initial residual,
// a BiCG step along M^-1 p and a minimal-residual step along M^-1 s per
// iteration; stops on the recursive residual and reports the true one.  A
// vanishing <r^, r> restarts from the current iterate.
template <class T, class OpA, class OpM>
int bicgstab(amgt_ctx* ctx, int k, OpA apply_A, OpM apply_M, const T* b, T* x, bool x_zero,
             double tol, int maxit, KrylovResult& res, amgt_stats* st, double bnorm_in,
             int hist_base) {
  const long long n = ctx->lv[k].nsdof * ctx->lv[k].nadof();
  const size_t bytes = (size_t)n * sizeof(T);
  T *r, *rh, *p, *v, *s, *t, *ph, *sh;
  TRY(wsvec<T>(ctx, k, 8, &r));
  TRY(wsvec<T>(ctx, k, 9, &rh));
  TRY(wsvec<T>(ctx, k, 10, &p));
  TRY(wsvec<T>(ctx, k, 11, &v));
  TRY(wsvec<T>(ctx, k, 12, &s));
  TRY(wsvec<T>(ctx, k, 13, &t));
  TRY(wsvec<T>(ctx, k, 14, &ph));
  TRY(wsvec<T>(ctx, k, 15, &sh));
  double bnorm = bnorm_in;
  if (bnorm < 0) TRY(norm2<T>(ctx, b, n, &bnorm));
  res = KrylovResult();
  if (bnorm == 0.0) {
    CK(cudaMemsetAsync(x, 0, bytes, ctx->stream));
    return AMGT_OK;
  }
  res.cycles = 1;
  if (!std::isfinite(bnorm)) return fail(ctx, AMGT_ERR_NAN, "right-hand side is not finite");
  auto residual = [&]() -> int {  // r = b - A x
    if (x_zero) {
      CK(cudaMemcpyAsync(r, b, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      CK(cudaMemsetAsync(x, 0, bytes, ctx->stream));
      x_zero = false;
    } else {
      TRY(apply_A(x, r));
      launch_axpby<T>(n, 1.0, b, -1.0, r, ctx->stream);
    }
    return AMGT_OK;
  };
  TRY(residual());
  double rr;
  TRY(norm2<T>(ctx, r, n, &rr));
  res.relres = rr / bnorm;
  double rho_old = 1.0, alpha = 1.0, omega = 1.0;
  bool fresh = true;  // shadow residual and directions to (re)set
  while (res.relres >= tol && res.its < maxit) {
    if (fresh) {
      CK(cudaMemcpyAsync(rh, r, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      CK(cudaMemsetAsync(p, 0, bytes, ctx->stream));
      CK(cudaMemsetAsync(v, 0, bytes, ctx->stream));
      rho_old = alpha = omega = 1.0;
      fresh = false;
    }
    double rho;
    TRY(dots_with<T>(ctx, n, {rh}, r, &rho));
    if (!std::isfinite(rho)) return fail(ctx, AMGT_ERR_NAN, "BiCGStab inner product is not finite");
    if (rho == 0.0) {
      fresh = true;
      continue;
    }
    const double beta = (rho / rho_old) * (alpha / omega);
    launch_axpby<T>(n, -omega, v, 1.0, p, ctx->stream);  // p = r + beta (p - omega v)
    launch_axpby<T>(n, 1.0, r, beta, p, ctx->stream);
    TRY(apply_M(p, ph));
    TRY(apply_A(ph, v));
    double rhv;
    TRY(dots_with<T>(ctx, n, {rh}, v, &rhv));
    if (rhv == 0.0) return fail(ctx, AMGT_ERR_BREAKDOWN, "BiCGStab: <r^, v> = 0");
    alpha = rho / rhv;
    launch_scale_copy<T>(n, 1.0, r, s, ctx->stream);  // s = r - alpha v
    launch_axpby<T>(n, -alpha, v, 1.0, s, ctx->stream);
    double ss;
    TRY(dots_with<T>(ctx, n, {s}, s, &ss));
    res.its++;
    const double srel = std::sqrt(std::max(ss, 0.0)) / bnorm;
    if (srel < tol) {
      launch_axpby<T>(n, alpha, ph, 1.0, x, ctx->stream);
      res.relres = srel;
      if (st && hist_base + res.its - 1 < AMGT_MAX_HIST) {
        st->hist[hist_base + res.its - 1] = srel;
        st->nhist = hist_base + res.its;
      }
      break;
    }
    TRY(apply_M(s, sh));
    TRY(apply_A(sh, t));
    double ts[2];
    TRY(dots_with<T>(ctx, n, {s, t}, t, ts));  // <s, t>, <t, t>
    if (ts[1] == 0.0) return fail(ctx, AMGT_ERR_BREAKDOWN, "BiCGStab: t = 0");
    omega = ts[0] / ts[1];
    launch_axpby<T>(n, alpha, ph, 1.0, x, ctx->stream);  // x += alpha ph + omega sh
    launch_axpby<T>(n, omega, sh, 1.0, x, ctx->stream);
    launch_scale_copy<T>(n, 1.0, s, r, ctx->stream);  // r = s - omega t
    launch_axpby<T>(n, -omega, t, 1.0, r, ctx->stream);
    TRY(dots_with<T>(ctx, n, {r}, r, &rr));
    res.relres = std::sqrt(std::max(rr, 0.0)) / bnorm;
    if (!std::isfinite(res.relres)) return fail(ctx, AMGT_ERR_NAN, "residual is not finite");
    if (st && hist_base + res.its - 1 < AMGT_MAX_HIST) {
      st->hist[hist_base + res.its - 1] = res.relres;
      st->nhist = hist_base + res.its;
    }
    rho_old = rho;
    if (omega == 0.0) fresh = true;
  }
  // the true residual decides
  TRY(residual());
  TRY(norm2<T>(ctx, r, n, &rr));
  res.relres = rr / bnorm;
  return AMGT_OK;
}

}  // namespace

// =================================================================== C ABI
namespace {
struct TuneChoice {
  int G = 0, stages = 0, gs_kernel = 0;
};
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune_cache;

// seconds per call of fn() on the context's stream (events, after one warm-up)
template <class F>
int time_on_stream(amgt_ctx* ctx, int reps, F fn, double* sec) {
  TRY(fn());
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  CK(cudaEventRecord(a, ctx->stream));
  for (int r = 0; r < reps; ++r) {
    const int rc = fn();
    if (rc != AMGT_OK) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return rc;
    }
  }
  CK(cudaEventRecord(b, ctx->stream));
  CK(cudaEventSynchronize(b));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *sec = ms / 1e3 / reps;
  return AMGT_OK;
}
}  // namespace

extern "C" {

int amgt_create(amgt_ctx** out, int device, void* stream) {
  if (!out) return AMGT_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return AMGT_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return AMGT_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return AMGT_ERR_CUDA;
  auto* ctx = new amgt_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  *out = ctx;
  return AMGT_OK;
}

void amgt_destroy(amgt_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
}

const char* amgt_last_error(const amgt_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

int amgt_set_stream(amgt_ctx* ctx, void* stream) {
  if (!ctx) return AMGT_ERR_ARG;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return AMGT_OK;
}

int amgt_query_launches(int64_t* count) {
  if (!count) return AMGT_ERR_ARG;
  *count = launch_count();
  return AMGT_OK;
}

int amgt_query_kernel_stats(amgt_ctx* ctx, int kernel, int reset, double* ms, int64_t* launches,
                            double* work) {
  if (!ctx) return AMGT_ERR_ARG;
  if (kernel < 0 || kernel >= AMGT_KT_COUNT) return fail(ctx, AMGT_ERR_ARG, "unknown kernel id");
  for (auto& p : ctx->kt_pending) {
    CK(cudaEventSynchronize(p.b));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, p.a, p.b));
    ctx->kt_ms[p.id] += t;
    ctx->kt_n[p.id] += 1;
    ctx->kt_work[p.id] += p.work;
    ctx->kt_free.push_back(p.a);
    ctx->kt_free.push_back(p.b);
  }
  ctx->kt_pending.clear();
  if (ms) *ms = ctx->kt_ms[kernel];
  if (launches) *launches = ctx->kt_n[kernel];
  if (work) *work = ctx->kt_work[kernel];
  if (reset) {
    ctx->kt_ms[kernel] = 0.0;
    ctx->kt_n[kernel] = 0;
    ctx->kt_work[kernel] = 0.0;
  }
  return AMGT_OK;
}

int amgt_query_kernel_time(amgt_ctx* ctx, int kernel, int reset, double* ms, int64_t* launches) {
  return amgt_query_kernel_stats(ctx, kernel, reset, ms, launches, nullptr);
}

int amgt_sync(amgt_ctx* ctx) {
  if (!ctx) return AMGT_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->d_status) {
    int st = 0;
    CK(cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
      CK(cudaMemset(ctx->d_status, 0, sizeof(int)));
      return fail(ctx, AMGT_ERR_DEVICE_TIMEOUT,
                  "a bounded device-side wait gave up (code " + std::to_string(st) + ")");
    }
  }
  return AMGT_OK;
}

int amgt_set_mesh_cartesian(amgt_ctx* ctx, int dim, const int64_t ncell[3], const double lo[3],
                            const double hi[3]) {
  if (!ctx) return AMGT_ERR_ARG;
  if ((dim != 2 && dim != 3) || !ncell || !lo || !hi) return fail(ctx, AMGT_ERR_ARG, "bad mesh");
  for (int e = 0; e < dim; ++e) {
    if (ncell[e] < 1 || ncell[e] > 2047) return fail(ctx, AMGT_ERR_ARG, "cells per axis must be 1..2047");
    if (!(hi[e] > lo[e])) return fail(ctx, AMGT_ERR_ARG, "hi must exceed lo");
  }
  ctx->dim = dim;
  for (int e = 0; e < 3; ++e) {
    ctx->ncell[e] = e < dim ? ncell[e] : 1;
    ctx->lo[e] = lo[e];
    ctx->hi[e] = hi[e];
  }
  ctx->sigma_t.clear();
  ctx->sigma_s.clear();
  ctx->qsrc.clear();
  ctx->N = -1;
  ctx->dirty = true;
  return AMGT_OK;
}

int amgt_set_materials(amgt_ctx* ctx, const double* st, const double* ss, const int32_t* mat_id,
                       int nmat, int N, const double* f) {
  if (!ctx) return AMGT_ERR_ARG;
  if (ctx->dim == 0) return fail(ctx, AMGT_ERR_STATE, "set the mesh first");
  if (!st || !ss || !f || N < 0 || N > 128 || nmat < 1 || (!mat_id && nmat != 1))
    return fail(ctx, AMGT_ERR_ARG,
                "bad materials: need sigma_t, sigma_s, f, 0 <= N <= 128, nmat >= 1 (1 without "
                "mat_id)");
  const int64_t C = ctx->ncell[0] * ctx->ncell[1] * ctx->ncell[2];
  for (int64_t c = 0; c < C; ++c) {
    if (!(st[c] > 0.0) || !(ss[c] >= 0.0) || !std::isfinite(st[c]) || !std::isfinite(ss[c]))
      return fail(ctx, AMGT_ERR_ARG, "need sigma_t > 0 and sigma_s >= 0, finite");
    if (mat_id && (mat_id[c] < 0 || mat_id[c] >= nmat))
      return fail(ctx, AMGT_ERR_ARG, "mat_id out of range");
  }
  for (int64_t i = 0; i < (int64_t)nmat * (N + 1); ++i)
    if (!std::isfinite(f[i])) return fail(ctx, AMGT_ERR_ARG, "moments are not finite");
  for (int m = 0; m < nmat; ++m)
    if (std::fabs(f[(size_t)m * (N + 1)] - 1.0) > 1e-12)
      return fail(ctx, AMGT_ERR_ARG, "f[m][0] must be 1 (sigma_s is the n = 0 moment)");
  ctx->sigma_t.assign(st, st + C);
  ctx->sigma_s.assign(ss, ss + C);
  ctx->ftab.assign(f, f + (size_t)nmat * (N + 1));
  ctx->nf = nmat;
  if (nmat > 1)
    ctx->fid.assign(mat_id, mat_id + C);
  else
    ctx->fid.clear();
  ctx->N = N;
  ctx->dirty = true;
  return AMGT_OK;
}

int amgt_set_angular_uniform(amgt_ctx* ctx, int basis, int level) {
  if (!ctx) return AMGT_ERR_ARG;
  if ((basis != 0 && basis != 1) || level < 0 || level > 7)
    return fail(ctx, AMGT_ERR_ARG, "basis 0/1 and level 0..7");
  ctx->basis = basis;
  ctx->paths = uniform_paths(level);
  ctx->dirty = true;
  return AMGT_OK;
}

int amgt_set_angular_aniso(amgt_ctx* ctx, int basis, const double axis[3], int lmax) {
  if (!ctx) return AMGT_ERR_ARG;
  if ((basis != 0 && basis != 1) || lmax < 0 || lmax > 8 || !axis)
    return fail(ctx, AMGT_ERR_ARG, "basis 0/1, lmax 0..8, axis non-null");
  if (axis[0] == 0 && axis[1] == 0 && axis[2] == 0) return fail(ctx, AMGT_ERR_ARG, "zero axis");
  ctx->basis = basis;
  ctx->paths = aniso_paths(lmax, axis);
  ctx->dirty = true;
  return AMGT_OK;
}

int amgt_set_multigrid(amgt_ctx* ctx, int nlevels, const int* Nr, int nu_pre, int nu_post,
                       int coarse_sweeps) {
  if (!ctx) return AMGT_ERR_ARG;
  if (nlevels < 1 || nlevels > 9 || nu_pre < 0 || nu_post < 0 || coarse_sweeps < 0)
    return fail(ctx, AMGT_ERR_ARG, "bad multigrid parameters");
  ctx->nlevels = nlevels;
  ctx->Nr.clear();
  if (Nr)
    for (int i = 0; i < nlevels; ++i) {
      if (Nr[i] < 0) return fail(ctx, AMGT_ERR_ARG, "negative scatter order");
      ctx->Nr.push_back(Nr[i]);
    }
  ctx->nu_pre = nu_pre;
  ctx->nu_post = nu_post;
  ctx->coarse_sweeps = coarse_sweeps;
  ctx->dirty = true;
  return AMGT_OK;
}

int amgt_set_source_iso(amgt_ctx* ctx, const double* q) {
  if (!ctx) return AMGT_ERR_ARG;
  if (ctx->dim == 0) return fail(ctx, AMGT_ERR_STATE, "set the mesh first");
  if (!q) return fail(ctx, AMGT_ERR_ARG, "null source");
  const int64_t C = ctx->ncell[0] * ctx->ncell[1] * ctx->ncell[2];
  for (int64_t c = 0; c < C; ++c)
    if (!std::isfinite(q[c])) return fail(ctx, AMGT_ERR_ARG, "source is not finite");
  ctx->qsrc.assign(q, q + C);
  if (!ctx->dirty && ctx->d_q) {
    // ordered on the context's stream; returns once the host data is staged
    CK(cudaMemcpyAsync(ctx->d_q, ctx->qsrc.data(), sizeof(double) * C, cudaMemcpyHostToDevice,
                       ctx->stream));
  } else {
    ctx->dirty = true;
  }
  return AMGT_OK;
}

int amgt_set_boundary(amgt_ctx* ctx, int face, int kind, const double* params) {
  if (!ctx) return AMGT_ERR_ARG;
  if (face < 0 || face >= 6 || kind < 0 || kind > 3)
    return fail(ctx, AMGT_ERR_ARG,
                "face 0..5, kind 0 (vacuum), 1 (isotropic inflow), 2 (normal pencil beam) or 3 "
                "(pencil beam of any inward direction over part of the face)");
  if (kind != 0 && !params) return fail(ctx, AMGT_ERR_ARG, "inflow needs params");
  const int np = kind == 3 ? 8 : (kind != 0 ? 1 : 0);
  for (int i = 0; i < np; ++i)
    if (!std::isfinite(params[i])) return fail(ctx, AMGT_ERR_ARG, "boundary value is not finite");
  if (kind == 3) {
    const double* d = params + 1;
    const double nrm = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(nrm > 0.0)) return fail(ctx, AMGT_ERR_ARG, "beam direction is zero");
    const double nsgn = (face & 1) ? 1.0 : -1.0;  // outward normal along axis face / 2
    if (!(d[face / 2] / nrm * nsgn < -1e-12))
      return fail(ctx, AMGT_ERR_ARG, "beam direction must point into the domain");
    if (!(params[4] < params[5]) || (ctx->dim == 3 && !(params[6] < params[7])))
      return fail(ctx, AMGT_ERR_ARG, "beam range needs u0 < u1 (and v0 < v1 in 3D)");
    for (int e = 0; e < 3; ++e) ctx->bdir[face][e] = d[e] / nrm;
    for (int e = 0; e < 4; ++e) ctx->brange[face][e] = params[4 + e];
  }
  ctx->bkind[face] = kind;
  ctx->bval[face] = kind != 0 ? params[0] : 0.0;
  ctx->dirty = true;
  return AMGT_OK;
}

int amgt_set_adjoint(amgt_ctx* ctx, int adjoint) {
  if (!ctx) return AMGT_ERR_ARG;
  if (adjoint != 0 && adjoint != 1) return fail(ctx, AMGT_ERR_ARG, "adjoint 0 or 1");
  if ((adjoint == 1) != ctx->adjoint) ctx->dirty = true;
  ctx->adjoint = adjoint == 1;
  return AMGT_OK;
}

int amgt_response(amgt_ctx* ctx, int device, const double* psi, double* R) {
  if (!ctx || !psi || !R) return AMGT_ERR_ARG;
  TRY(build(ctx));
  const Level& L0 = ctx->lv[0];
  const long long n = L0.nsdof * L0.nadof();
  double *g, *x;
  TRY(wsvec<double>(ctx, 0, 7, &g));
  TRY(source_impl<double>(ctx, 0, g));
  if (device) {
    x = const_cast<double*>(psi);
  } else {
    TRY(wsvec<double>(ctx, 0, 5, &x));
    CK(cudaMemcpyAsync(x, psi, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  }
  const int nblk = gemv_blocks(n);
  void** slot = ctx->d_ptrs + 200;
  const double* gp = g;
  CK(cudaMemcpyAsync(slot, &gp, sizeof(void*), cudaMemcpyHostToDevice, ctx->stream));
  launch_multidot<double>(n, 1, reinterpret_cast<const double* const*>(slot), x, ctx->d_partials,
                          nblk, ctx->d_dots, ctx->stream);
  CK(cudaGetLastError());
  TRY(dev_dots<double>(ctx, 1, R));
  return AMGT_OK;
}

int amgt_response_gradients(amgt_ctx* ctx, int device, const double* psi, const double* lambda,
                            double* dsigma_t, double* dsigma_s, double* dfmom) {
  if (!ctx || !psi || !lambda || !dsigma_t || !dsigma_s || !dfmom) return AMGT_ERR_ARG;
  TRY(build(ctx));
  const Level& L0 = ctx->lv[0];
  const long long n = L0.nsdof * L0.nadof();
  const int C = ctx->geom.C, nm = L0.nmom, N = L0.Nr;
  const int nf = ctx->nf;
  if ((int)ctx->ftab.size() < nf * (ctx->N + 1))
    return fail(ctx, AMGT_ERR_STATE, "Legendre moments not set");
  const double *p, *l;
  if (device) {
    p = psi;
    l = lambda;
  } else {
    double *pp, *ll;
    TRY(wsvec<double>(ctx, 0, 5, &pp));
    TRY(wsvec<double>(ctx, 0, 6, &ll));
    CK(cudaMemcpyAsync(pp, psi, (size_t)n * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ll, lambda, (size_t)n * 8, cudaMemcpyHostToDevice, ctx->stream));
    p = pp;
    l = ll;
  }
  // scratch: both moment sets, the outputs, f_n
  const size_t need = ((size_t)2 * L0.nsdof * nm + 2 * (size_t)C + 2 * (size_t)nf * (N + 1)) * 8;
  if (ctx->grad_bytes < need) {
    double* q;
    TRY(dalloc<double>(ctx, need / 8, &q));
    ctx->d_grad = q;
    ctx->grad_bytes = need;
  }
  double* PhiP = ctx->d_grad;
  double* PhiL = PhiP + (size_t)L0.nsdof * nm;
  double* dt = PhiL + (size_t)L0.nsdof * nm;
  double* ds = dt + C;
  double* df = ds + C;
  double* fm = df + (size_t)nf * (N + 1);
  // the shapes at the finest level's order N (= the problem's order)
  std::vector<double> fl((size_t)nf * (N + 1));
  for (int m = 0; m < nf; ++m)
    for (int n2 = 0; n2 <= N; ++n2) fl[(size_t)m * (N + 1) + n2] = ctx->ftab[(size_t)m * (ctx->N + 1) + n2];
  CK(cudaMemcpyAsync(fm, fl.data(), fl.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(df, 0, (size_t)nf * (N + 1) * 8, ctx->stream));
  GemmEpi e0{};
  e0.mode = 0;
  launch_gemm<double>((int)L0.nsdof, nm, L0.nadof(), p, L0.nadof(), L0.d64.X, nm, PhiP, nm, e0,
                      ctx->stream);
  launch_gemm<double>((int)L0.nsdof, nm, L0.nadof(), l, L0.nadof(), L0.d64.X, nm, PhiL, nm, e0,
                      ctx->stream);
  const Geom g = level_geom(ctx, 0);
  launch_grad_sigma_t(g, L0.d64.Mang, p, l, dt, ctx->stream);
  launch_grad_moments(g, nm, N, PhiP, PhiL, fm, nf > 1 ? ctx->d_fid : nullptr, ctx->d_sigs, ds,
                      df, ctx->stream);
  CK(cudaGetLastError());
  const cudaMemcpyKind kind = device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(dsigma_t, dt, (size_t)C * 8, kind, ctx->stream));
  CK(cudaMemcpyAsync(dsigma_s, ds, (size_t)C * 8, kind, ctx->stream));
  CK(cudaMemcpyAsync(dfmom, df, (size_t)nf * (N + 1) * 8, kind, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return AMGT_OK;
}

// ---- batched solves and autotuning

// A batch's contexts are non-null and distinct: two host threads driving one
// context would race on its workspaces and stream.
static bool batch_contexts_ok(amgt_ctx* const* ctxs, int n) {
  std::vector<amgt_ctx*> v(ctxs, ctxs + n);
  if (std::find(v.begin(), v.end(), nullptr) != v.end()) return false;
  std::sort(v.begin(), v.end());
  return std::adjacent_find(v.begin(), v.end()) == v.end();
}

int amgt_solve_batch(amgt_ctx* const* ctxs, int n, const amgt_options* opt, double* const* psi,
                     double* const* phi, amgt_stats* stats, int nthreads) {
  if (!ctxs || n < 0 || !opt || !psi || !batch_contexts_ok(ctxs, n)) return AMGT_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!psi[i]) return AMGT_ERR_ARG;
  int nt = nthreads > 0 ? nthreads : std::min(n, 16);
  nt = std::max(1, std::min(nt, std::max(1, n)));
  std::vector<int> rc(n, AMGT_OK);
  std::atomic<int> next{0};
  auto work = [&] {
    for (int i; (i = next.fetch_add(1)) < n;) {
      cudaSetDevice(ctxs[i]->device);
      rc[i] = amgt_solve(ctxs[i], opt, nullptr, psi[i], phi ? phi[i] : nullptr,
                         stats ? &stats[i] : nullptr);
      // a bounded device wait that gave up is reported with the solve
      const int rs = amgt_sync(ctxs[i]);
      if (rc[i] == AMGT_OK) rc[i] = rs;
    }
  };
  std::vector<std::thread> ts;
  for (int t = 0; t < nt; ++t) ts.emplace_back(work);
  for (auto& t : ts) t.join();
  for (int i = 0; i < n; ++i)
    if (rc[i] != AMGT_OK) return rc[i];
  return AMGT_OK;
}

int amgt_setup_batch(amgt_ctx* const* ctxs, int n, int nthreads) {
  if (!ctxs || n < 0 || !batch_contexts_ok(ctxs, n)) return AMGT_ERR_ARG;
  int nt = nthreads > 0 ? nthreads : std::min(n, 16);
  nt = std::max(1, std::min(nt, std::max(1, n)));
  std::vector<int> rc(n, AMGT_OK);
  std::atomic<int> next{0};
  auto work = [&] {
    for (int i; (i = next.fetch_add(1)) < n;) {
      cudaSetDevice(ctxs[i]->device);
      rc[i] = build(ctxs[i]);
      if (rc[i] == AMGT_OK && cudaStreamSynchronize(ctxs[i]->stream) != cudaSuccess) {
        cudaGetLastError();
        rc[i] = fail(ctxs[i], AMGT_ERR_CUDA, "set-up did not complete");
      }
    }
  };
  std::vector<std::thread> ts;
  for (int t = 0; t < nt; ++t) ts.emplace_back(work);
  for (auto& t : ts) t.join();
  for (int i = 0; i < n; ++i)
    if (rc[i] != AMGT_OK) return rc[i];
  return AMGT_OK;
}

int amgt_autotune(amgt_ctx* ctx, int what, int* choice) {
  if (!ctx) return AMGT_ERR_ARG;
  TRY(build(ctx));
  drop_graphs(ctx);
  const Geom g0 = level_geom(ctx, 0);
  const int nl = (int)ctx->lv.size();
  std::string key = std::to_string(g0.dim) + "/" + std::to_string(g0.nx) + "x" +
                    std::to_string(g0.ny) + "x" + std::to_string(g0.nz) + "/" +
                    std::to_string(ctx->basis);
  for (int k = 0; k < nl; ++k) key += "/" + std::to_string(ctx->lv[k].mesh.P) + ":" + std::to_string(ctx->lv[k].nmom);
  key += "/" + std::to_string(std::min(ctx->nmat, 64)) + "/" + std::to_string(ctx->nf);
  TuneChoice best;
  bool cached = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      best = it->second;
      cached = true;
    }
  }
  float *x, *y;
  TRY(wsvec<float>(ctx, 0, 3, &x));
  TRY(wsvec<float>(ctx, 0, 4, &y));
  if (!cached) {
    CK(cudaMemsetAsync(x, 0, (size_t)ctx->lv[0].nsdof * ctx->lv[0].nadof() * 4, ctx->stream));
    best.G = ctx->sweep_group;
    best.stages = ctx->sweep_stages;
    best.gs_kernel = ctx->gs_kernel;
    if (what & 1) {
      // sweep: patches per block (all levels) and, in 2D, the copy depth
      double tbest = 1e30;
      const std::vector<int> Gs = g0.dim == 2 ? std::vector<int>{1, 2, 4, 8}
                                              : std::vector<int>{1, 2, 4, 8, 16};
      const std::vector<int> Ss = g0.dim == 2 ? std::vector<int>{3, 4} : std::vector<int>{0};
      for (int G : Gs) {
        if (g0.dim == 2 && g0.ny * G > 512) continue;
        ctx->sweep_group = G;
        for (int k = 0; k < nl; ++k) TRY(make_sweep_tasks(ctx, ctx->lv[k], level_geom(ctx, k), G));
        for (int st : Ss) {
          ctx->sweep_stages = st;
          double t;
          TRY(time_on_stream(ctx, 3, [&] { return sweep_impl<float>(ctx, 0, x, y); }, &t));
          if (t < tbest) {
            tbest = t;
            best.G = G;
            best.stages = st;
          }
        }
      }
    }
    if (what & 2) {
      // coarse solver: row-pipelined, thread-group (cluster) and warp kernels
      const Level& Lc = ctx->lv[nl - 1];
      float *fc, *xc;
      TRY(wsvec<float>(ctx, nl - 1, 3, &fc));
      TRY(wsvec<float>(ctx, nl - 1, 4, &xc));
      CK(cudaMemsetAsync(fc, 0, (size_t)Lc.nsdof * Lc.nadof() * 4, ctx->stream));
      double tbest = 1e30;
      const std::vector<int> cand =
          store<float>(Lc).TinvT ? std::vector<int>{6, 3} : std::vector<int>{2, 1};
      for (int v : cand) {
        if (v == 6 && Lc.rows_nb == 0) continue;
        ctx->gs_kernel = v;
        double t;
        const int rc = time_on_stream(ctx, 1, [&] { return coarse_gs_impl<float>(ctx, 1, fc, xc); }, &t);
        if (rc != AMGT_OK) continue;
        if (t < tbest) {
          tbest = t;
          best.gs_kernel = v;
        }
      }
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
  }
  ctx->sweep_group = best.G;
  ctx->sweep_stages = best.stages;
  ctx->gs_kernel = best.gs_kernel;
  for (int k = 0; k < nl; ++k) TRY(make_sweep_tasks(ctx, ctx->lv[k], level_geom(ctx, k), best.G));
  if (choice) {
    choice[0] = best.G;
    choice[1] = best.stages;
    choice[2] = best.gs_kernel;
    choice[3] = cached ? 1 : 0;
  }
  return AMGT_OK;
}

int amgt_set_tuning(amgt_ctx* ctx, int key, int value) {
  if (!ctx) return AMGT_ERR_ARG;
  drop_graphs(ctx);  // a captured cycle holds the old choices
  if (key == AMGT_TUNE_GS_KERNEL) {
    if (value < 0 || value > 6) return fail(ctx, AMGT_ERR_ARG, "GS kernel 0..6");
    ctx->gs_kernel = value;
    return AMGT_OK;
  }
  if (key == AMGT_TUNE_GS_CLUSTER) {
    if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16)
      return fail(ctx, AMGT_ERR_ARG, "cluster size 0, 1, 2, 4, 8 or 16");
    ctx->gs_cluster_size = value;
    return AMGT_OK;
  }
  if (key == AMGT_TUNE_GS_GRID_BLOCKS) {
    if (value < 0 || value > 4096) return fail(ctx, AMGT_ERR_ARG, "grid blocks 0..4096");
    if (value != ctx->gs_grid_blocks) ctx->dirty = true;  // the row tables depend on it
    ctx->gs_grid_blocks = value;
    return AMGT_OK;
  }
  if (key == AMGT_TUNE_GRAPHS) {
    if (value != 0 && value != 1) return fail(ctx, AMGT_ERR_ARG, "graphs 0 or 1");
    ctx->use_graphs = value == 1;
    drop_graphs(ctx);
    return AMGT_OK;
  }
  if (key == AMGT_TUNE_GS_FORM) {
    if (value < 0 || value > 2) return fail(ctx, AMGT_ERR_ARG, "GS form 0, 1 or 2");
    if (value != ctx->gs_form) ctx->dirty = true;  // the row plan depends on it
    ctx->gs_form = value;
    return AMGT_OK;
  }
  if (key == AMGT_TUNE_COARSE_F64) {
    if (value != 0 && value != 1) return fail(ctx, AMGT_ERR_ARG, "coarse FP64 0 or 1");
    ctx->coarse_f64 = value;
    return AMGT_OK;
  }
  if (key == AMGT_TUNE_TEST_SWEEP_HOLD) {
    if (value != 0 && value != 1) return fail(ctx, AMGT_ERR_ARG, "test sweep hold 0 or 1");
    ctx->test_sweep_hold = value;
    return AMGT_OK;
  }
  if (key == AMGT_TUNE_F32_SCATTER) {
    if (value != 0 && value != 1) return fail(ctx, AMGT_ERR_ARG, "FP32 scatter 0 or 1");
    ctx->f32_scatter = value;
    return AMGT_OK;
  }
  if (key == AMGT_TUNE_FP64_SCATTER) {
    if (value < 0 || value > 2) return fail(ctx, AMGT_ERR_ARG, "FP64 scatter 0, 1 or 2");
    ctx->fp64_scatter = value;
    return AMGT_OK;
  }
  if (key == AMGT_TUNE_SWEEP_KERNEL) {
    if (value < 0 || value > 2) return fail(ctx, AMGT_ERR_ARG, "sweep kernel 0, 1 or 2");
    ctx->sweep_kernel = value;
    return AMGT_OK;
  }
  if (key == AMGT_TUNE_SPLIT_ROWS) {
    if (value < 0) return fail(ctx, AMGT_ERR_ARG, "split rows >= 0");
    ctx->split_rows = value;
    return AMGT_OK;
  }
  if (key == AMGT_TUNE_KERNEL_TIMERS) {
    if (value != 0 && value != 1) return fail(ctx, AMGT_ERR_ARG, "kernel timers 0 or 1");
    ctx->ktimers = value == 1;
    return AMGT_OK;
  }
  if (key == AMGT_TUNE_SWEEP_STAGES) {
    if (value < 0 || value > 6) return fail(ctx, AMGT_ERR_ARG, "sweep stages 0..6");
    ctx->sweep_stages = value;
    return AMGT_OK;
  }
  if (key == AMGT_TUNE_SWEEP_GROUP) {
    if (value < 0 || value > 16) return fail(ctx, AMGT_ERR_ARG, "sweep group 0..16");
    if (value != ctx->sweep_group) ctx->dirty = true;
    ctx->sweep_group = value;
    return AMGT_OK;
  }
  return fail(ctx, AMGT_ERR_ARG, "unknown tuning key");
}

int amgt_query_sizes(const amgt_ctx* cctx, int level, int64_t* nsdof, int64_t* nadof) {
  amgt_ctx* ctx = const_cast<amgt_ctx*>(cctx);
  if (!ctx) return AMGT_ERR_ARG;
  TRY(check_level(ctx, level));
  if (nsdof) *nsdof = ctx->lv[level].nsdof;
  if (nadof) *nadof = ctx->lv[level].nadof();
  return AMGT_OK;
}

#define DISPATCH(dtype, CALL64, CALL32)                                            \
  do {                                                                            \
    if ((dtype) == AMGT_F64 || (dtype) == AMGT_F64_SPLIT) return CALL64;          \
    if ((dtype) == AMGT_F32 || (dtype) == AMGT_F32_BF16TC || (dtype) == AMGT_F32_TC3) \
      return CALL32;                                                              \
    return fail(ctx, AMGT_ERR_ARG,                                                \
                "dtype must be AMGT_F64, AMGT_F64_SPLIT, AMGT_F32, AMGT_F32_BF16TC or " \
                "AMGT_F32_TC3");                                                  \
  } while (0)

namespace {
// scatter path of an FP32 dtype (see scatter_impl)
int f32_path(int dtype) {
  return dtype == AMGT_F32_BF16TC ? 1 : dtype == AMGT_F32_TC3 ? 2 : 0;
}
}  // namespace

int amgt_op_source(amgt_ctx* ctx, int level, int dtype, void* f) {
  if (!ctx) return AMGT_ERR_ARG;
  TRY(check_level(ctx, level));
  DISPATCH(dtype, source_impl<double>(ctx, level, (double*)f),
           source_impl<float>(ctx, level, (float*)f));
}

int amgt_op_sweep(amgt_ctx* ctx, int level, int dtype, const void* b, void* psi) {
  if (!ctx) return AMGT_ERR_ARG;
  TRY(check_level(ctx, level));
  if (b == psi) return fail(ctx, AMGT_ERR_ARG, "sweep input and output must not alias");
  DISPATCH(dtype, sweep_impl<double>(ctx, level, (const double*)b, (double*)psi),
           sweep_impl<float>(ctx, level, (const float*)b, (float*)psi));
}

int amgt_op_apply_L(amgt_ctx* ctx, int level, int dtype, const void* x, void* y) {
  if (!ctx) return AMGT_ERR_ARG;
  TRY(check_level(ctx, level));
  if (dtype == AMGT_F64_SPLIT)
    return applyL_df(ctx, level, 1.0, 0.0, (const double*)x, (double*)y);
  DISPATCH(dtype, applyL_impl<double>(ctx, level, 1.0, 0.0, (const double*)x, (double*)y),
           applyL_impl<float>(ctx, level, 1.0f, 0.0f, (const float*)x, (float*)y));
}

int amgt_op_scatter(amgt_ctx* ctx, int level, int dtype, const void* x, void* y) {
  if (!ctx) return AMGT_ERR_ARG;
  TRY(check_level(ctx, level));
  DISPATCH(dtype,
           scatter_impl<double>(ctx, level, dtype == AMGT_F64_SPLIT, (const double*)x, (double*)y, 1.0, 0.0, nullptr),
           scatter_impl<float>(ctx, level, f32_path(dtype), (const float*)x, (float*)y,
                               1.0, 0.0, nullptr));
}

int amgt_op_apply_A(amgt_ctx* ctx, int level, int dtype, const void* x, void* y) {
  if (!ctx) return AMGT_ERR_ARG;
  TRY(check_level(ctx, level));
  DISPATCH(dtype, applyA_impl<double>(ctx, level, dtype == AMGT_F64_SPLIT, (const double*)x, (double*)y),
           applyA_impl<float>(ctx, level, f32_path(dtype), (const float*)x, (float*)y));
}

int amgt_op_restrict(amgt_ctx* ctx, int level, int dtype, const void* rf, void* rc) {
  if (!ctx) return AMGT_ERR_ARG;
  TRY(check_level(ctx, level));
  if (level + 1 >= (int)ctx->lv.size()) return fail(ctx, AMGT_ERR_ARG, "no coarser level");
  DISPATCH(dtype, restrict_impl<double>(ctx, level, (const double*)rf, (double*)rc),
           restrict_impl<float>(ctx, level, (const float*)rf, (float*)rc));
}

int amgt_op_prolong(amgt_ctx* ctx, int level, int dtype, const void* xc, void* xf) {
  if (!ctx) return AMGT_ERR_ARG;
  TRY(check_level(ctx, level));
  if (level + 1 >= (int)ctx->lv.size()) return fail(ctx, AMGT_ERR_ARG, "no coarser level");
  DISPATCH(dtype, prolong_impl<double>(ctx, level, (const double*)xc, (double*)xf),
           prolong_impl<float>(ctx, level, (const float*)xc, (float*)xf));
}

int amgt_op_smooth(amgt_ctx* ctx, int level, int dtype, int nu, const void* f, void* phi) {
  if (!ctx) return AMGT_ERR_ARG;
  TRY(check_level(ctx, level));
  if (nu < 0) return fail(ctx, AMGT_ERR_ARG, "nu < 0");
  DISPATCH(dtype, smooth_impl<double>(ctx, level, dtype == AMGT_F64_SPLIT, nu, (const double*)f, (double*)phi, false),
           smooth_impl<float>(ctx, level, dtype == AMGT_F32_BF16TC, nu, (const float*)f,
                              (float*)phi, false));
}

int amgt_op_coarse_gs(amgt_ctx* ctx, int dtype, int sweeps, const void* f, void* phi) {
  if (!ctx) return AMGT_ERR_ARG;
  TRY(build(ctx));
  if (sweeps < 0) return fail(ctx, AMGT_ERR_ARG, "sweeps < 0");
  DISPATCH(dtype, coarse_gs_impl<double>(ctx, sweeps, (const double*)f, (double*)phi),
           coarse_gs_impl<float>(ctx, sweeps, (const float*)f, (float*)phi));
}

int amgt_op_coarse_gs_noalloc(amgt_ctx* ctx, int dtype, int sweeps, const void* f, void* phi) {
  if (!ctx) return AMGT_ERR_ARG;
  // set-up allocates, so it must already be complete
  if (ctx->dirty)
    return fail(ctx, AMGT_ERR_STATE,
                "problem set-up is not complete: call amgt_query_sizes (or any other "
                "operator) after the last set_* call first");
  if (sweeps < 0) return fail(ctx, AMGT_ERR_ARG, "sweeps < 0");
  if (f == phi) return fail(ctx, AMGT_ERR_ARG, "f and phi must not alias");
  DISPATCH(dtype, coarse_gs_noalloc_impl<double>(ctx, sweeps, (const double*)f, (double*)phi),
           coarse_gs_noalloc_impl<float>(ctx, sweeps, (const float*)f, (float*)phi));
}

int amgt_op_vcycle(amgt_ctx* ctx, int dtype, const void* f, void* phi) {
  if (!ctx) return AMGT_ERR_ARG;
  TRY(build(ctx));
  DISPATCH(dtype, vcycle_impl<double>(ctx, 0, dtype == AMGT_F64_SPLIT, (const double*)f, (double*)phi),
           vcycle_impl<float>(ctx, 0, dtype == AMGT_F32_BF16TC, (const float*)f, (float*)phi));
}

int amgt_op_scalar_flux(amgt_ctx* ctx, int level, int dtype, const void* psi, void* phi) {
  if (!ctx) return AMGT_ERR_ARG;
  TRY(check_level(ctx, level));
  DISPATCH(dtype, scalar_flux_impl<double>(ctx, level, (const double*)psi, (double*)phi),
           scalar_flux_impl<float>(ctx, level, (const float*)psi, (float*)phi));
}

int amgt_solve(amgt_ctx* ctx, const amgt_options* opt, const double* x0, double* psi,
               double* phi, amgt_stats* st) {
  if (!ctx) return AMGT_ERR_ARG;
  if (!opt || !psi) return fail(ctx, AMGT_ERR_ARG, "options and psi are required");
  if (opt->krylov != AMGT_KRYLOV_GMRES && opt->krylov != AMGT_KRYLOV_BICGSTAB)
    return fail(ctx, AMGT_ERR_ARG, "krylov: AMGT_KRYLOV_GMRES or AMGT_KRYLOV_BICGSTAB");
  TRY(build(ctx));
  const auto t0 = std::chrono::steady_clock::now();
  if (st) std::memset(st, 0, sizeof(*st));
  const Level& L0 = ctx->lv[0];
  const long long n = L0.nsdof * L0.nadof();
  const size_t bytes = (size_t)n * sizeof(double);
  const int m = opt->restart > 0 ? opt->restart : 20;
  const int maxit = opt->maxit > 0 ? opt->maxit : 1000;
  if (opt->precond == AMGT_PREC_MG && ctx->lv.size() < 2 && opt->mode == AMGT_MODE_F64) {
    // a one-level "cycle" is the coarse solver alone
  }
  double *b, *x;
  TRY(wsvec<double>(ctx, 0, 1, &b));
  if (opt->device_ptrs) {
    x = psi;
  } else {
    TRY(wsvec<double>(ctx, 0, 2, &x));
  }
  TRY(source_impl<double>(ctx, 0, b));
  bool x_zero = true;
  if (x0) {
    // x0 == psi on the device is a warm start in place: psi already holds it
    if (x0 != x)
      CK(cudaMemcpyAsync(x, x0, bytes, opt->device_ptrs ? cudaMemcpyDeviceToDevice
                                                        : cudaMemcpyHostToDevice, ctx->stream));
    x_zero = false;
  }
  KrylovResult kr;
  int rc = AMGT_OK;
  const int prec = opt->precond;
  // graphs and the per-kernel event timers exclude each other; the legacy
  // default stream cannot be captured
  const bool graphs = ctx->use_graphs && !ctx->ktimers && ctx->stream != nullptr &&
                      ctx->stream != cudaStreamLegacy && ctx->stream != cudaStreamPerThread;
  if (opt->mode == AMGT_MODE_F64) {
    const bool split = use_split64(ctx, false);
    auto A64 = [&](const double* xx, double* yy) { return applyA_impl<double>(ctx, 0, split, xx, yy); };
    auto M64 = [&](const double* v, double* z) -> int {
      if (prec == AMGT_PREC_SWEEP) return sweep_impl<double>(ctx, 0, v, z);
      if (prec == AMGT_PREC_MG)
        return graphs ? vcycle_graph<double>(ctx, split, v, z) : vcycle_impl<double>(ctx, 0, split, v, z);
      CK(cudaMemcpyAsync(z, v, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      return AMGT_OK;
    };
    if (opt->krylov == AMGT_KRYLOV_BICGSTAB)
      rc = bicgstab<double>(ctx, 0, A64, M64, b, x, x_zero, opt->tol, maxit, kr, st, -1.0, 0);
    else
      rc = gmres<double>(ctx, 0, A64, M64, b, x, x_zero, opt->tol, m, maxit, kr, st, -1.0, 0);
    if (st) {
      st->iterations = kr.its;
      st->outer_iterations = kr.cycles;
      st->relres = kr.relres;
    }
    if (rc == AMGT_OK && kr.relres >= opt->tol) rc = AMGT_ERR_NOT_CONVERGED;
  } else if (opt->mode == AMGT_MODE_MIXED) {
    const bool tc = tc_available();
    float *r32, *e32;
    double* r64;
    TRY(wsvec<double>(ctx, 0, 0, &r64));
    TRY(wsvec<float>(ctx, 0, 1, &r32));
    TRY(wsvec<float>(ctx, 0, 2, &e32));
    double bnorm;
    TRY(norm2<double>(ctx, b, n, &bnorm));
    if (!std::isfinite(bnorm)) return fail(ctx, AMGT_ERR_NAN, "right-hand side is not finite");
    if (bnorm == 0.0) {
      // b = 0: psi = 0 solves it exactly (relres 0, no iteration)
      CK(cudaMemsetAsync(x, 0, bytes, ctx->stream));
    }
    // the inner operator keeps FP32 accuracy (its rounding sets how far each
    // inner solve can go): the FP16 three-product tensor-core form, or the SIMT
    // FP32 contraction; the preconditioner's scatters use BF16 tensor cores
    const int a32_path = ctx->f32_scatter == 1 ? 0 : 2;
    // The Krylov method applies A to the preconditioner's output z, and z
    // left a sweep: L z = t exactly (the sweep inverts L), with t the sweep's
    // input (the sweep preconditioner) or the last post-smoothing sweep's
    // right-hand side S z' + f (workspace 3 of level 0, the V-cycle).  Then
    // A z = t - S z: one scatter and no L apply.
    const float* mz = nullptr;
    const float* mt = nullptr;
    auto A32 = [&](const float* xx, float* yy) -> int {
      if (xx == mz && mt) {
        mz = nullptr;
        return scatter_impl<float>(ctx, 0, a32_path, xx, yy, -1.0, 0.0, mt);
      }
      mz = nullptr;
      return applyA_impl<float>(ctx, 0, a32_path, xx, yy);
    };
    auto M32 = [&](const float* v, float* z) -> int {
      mz = nullptr;
      if (prec == AMGT_PREC_SWEEP) {
        TRY(sweep_impl<float>(ctx, 0, v, z));
        mz = z;
        mt = v;
        return AMGT_OK;
      }
      if (prec == AMGT_PREC_MG) {
        TRY(graphs ? vcycle_graph<float>(ctx, tc, v, z) : vcycle_impl<float>(ctx, 0, tc, v, z));
        if (ctx->lv.size() > 1 && ctx->nu_post >= 1) {
          float* t;
          TRY(wsvec<float>(ctx, 0, 3, &t));
          mz = z;
          mt = t;
        }
        return AMGT_OK;
      }
      CK(cudaMemcpyAsync(z, v, (size_t)n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
      return AMGT_OK;
    };
    int total_its = 0, outer = 0;
    double relres = bnorm > 0.0 ? 1.0 : 0.0;
    // inner tolerance: fixed, or aimed at the outer tolerance from the current
    // residual (the FP32 operator's rounding bounds how far one solve can go)
    auto inner_tol_for = [&](double rr) {
      if (opt->inner_tol > 0) return opt->inner_tol;
      return std::min(1e-2, std::max(3e-5, 0.3 * opt->tol / rr));
    };
    const int imax = opt->inner_maxit > 0 ? opt->inner_maxit : 200;
    // an adaptive inner solve that stalls above its target stops after two cycles
    const int imax_solve = opt->inner_tol > 0 ? imax : std::min(imax, 2 * m);
    while (bnorm > 0.0) {
      if (x_zero) {
        CK(cudaMemcpyAsync(r64, b, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      } else {
        // the refinement residual's operator: with the split-form scatter, L x
        // in double-float arithmetic (both ~1e-13, far below what 1e-8 needs)
        if (use_split64(ctx, true) && split_applies(ctx, 0)) {
          TRY(scatter_impl<double>(ctx, 0, 1, x, r64, -1.0, 0.0, nullptr));
          TRY(applyL_df(ctx, 0, 1.0, 1.0, x, r64));
        } else {
          TRY(applyA_impl<double>(ctx, 0, 0, x, r64));
        }
        launch_axpby<double>(n, 1.0, b, -1.0, r64, ctx->stream);
      }
      double rn;
      TRY(norm2<double>(ctx, r64, n, &rn));
      if (!std::isfinite(rn)) return fail(ctx, AMGT_ERR_NAN, "residual is not finite");
      relres = rn / bnorm;
      if (relres < opt->tol || total_its >= maxit || outer >= 50) break;
      launch_convert<double, float>(n, r64, r32, ctx->stream);
      launch_scale_copy<float>(n, 1.0 / rn, r32, r32, ctx->stream);
      KrylovResult ik;
      if (opt->krylov == AMGT_KRYLOV_BICGSTAB)
        rc = bicgstab<float>(ctx, 0, A32, M32, r32, e32, true, inner_tol_for(relres),
                             std::min(imax_solve, maxit - total_its), ik, st, 1.0, total_its);
      else
        rc = gmres<float>(ctx, 0, A32, M32, r32, e32, true, inner_tol_for(relres), m,
                          std::min(imax_solve, maxit - total_its), ik, st, 1.0, total_its);
      if (rc != AMGT_OK) break;
      total_its += ik.its;
      // x += rn * e  (FP64 accumulate)
      launch_convert<float, double>(n, e32, r64, ctx->stream);
      if (x_zero) {
        launch_scale_copy<double>(n, rn, r64, x, ctx->stream);
      } else {
        launch_axpby<double>(n, rn, r64, 1.0, x, ctx->stream);
      }
      x_zero = false;
      outer++;
      if (ik.its == 0) break;
    }
    if (st) {
      st->iterations = total_its;
      st->outer_iterations = outer;
      st->relres = relres;
    }
    if (rc == AMGT_OK && relres >= opt->tol) rc = AMGT_ERR_NOT_CONVERGED;
  } else {
    return fail(ctx, AMGT_ERR_ARG, "unknown mode");
  }
  if (rc != AMGT_OK && rc != AMGT_ERR_NOT_CONVERGED) return rc;
  if (phi) {
    double* ph;
    if (opt->device_ptrs) {
      ph = phi;
    } else {
      TRY(wsvec<double>(ctx, 0, 4, &ph));
    }
    TRY(scalar_flux_impl<double>(ctx, 0, x, ph));
    if (!opt->device_ptrs)
      CK(cudaMemcpyAsync(phi, ph, sizeof(double) * L0.nsdof, cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (!opt->device_ptrs) CK(cudaMemcpyAsync(psi, x, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (st)
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rc == AMGT_ERR_NOT_CONVERGED) ctx->err = "GMRES did not reach the tolerance within maxit";
  return rc;
}

}  // extern "C"
