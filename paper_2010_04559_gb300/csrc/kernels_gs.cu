// Coarse-angular-mesh solver (Sec. 4.2): block Gauss-Seidel sweeps over the
// (cell, patch) blocks in the sweep order, each block solve including the
// self-scatter and taking every other unknown at its latest value, with the
// scatter from the other patches of the cell evaluated through the cell's
// flux moments Phi_c[i][k] = sum_j psi[c*s+i][j] X[j][k]:
//
//   (K0_q + sigma_t kron(N, M_q) - sigma_s kron(N, S_qq)) x_q
//       = f_q - upwind_q + sigma_s N (X_q F Phi_c - S_qq x_q^old)
//   Phi_c += X_q^T (x_q - x_q^old)
//
// Order: sweep directions in index order; cells in upwind wavefront order;
// inside a cell the direction's patches in index order.  Cells of one
// wavefront level are independent (the scatter is cell-local), so they run
// concurrently: one warp per cell, all warps of one thread-block cluster, and
// a hardware cluster barrier between wavefront levels.
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <vector>
#include <mutex>

#include "gs_common.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace amgt {

// Fixed scratch for amgt_op_coarse_gs_noalloc: the cells' flux moments
// Phi[Nsdof][nmom] of the coarsest level.  It is part of the library image, so
// every GPU that loads the library holds it until the process exits.  All
// calls share it and it keeps the last call's contents; it is fully
// overwritten at the start of each call, so nothing needs clearing.
constexpr size_t kNoAllocMomentBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_moments[kNoAllocMomentBytes];

size_t noalloc_moment_bytes() { return kNoAllocMomentBytes; }

// Device address of g_noalloc_moments for `device`, looked up once per device
// with that device current (host code must not use the symbol itself as a
// device pointer).  Called at context set-up.
cudaError_t noalloc_moment_address(int device, void** out) {
  static std::mutex mu;
  static std::map<int, void*> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(device);
  if (it != cache.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return e;
  if (cur != device) {
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
  }
  void* ptr = nullptr;
  e = cudaGetSymbolAddress(&ptr, g_noalloc_moments);
  if (cur != device) cudaSetDevice(cur);
  if (e != cudaSuccess) return e;
  cache[device] = ptr;
  *out = ptr;
  return cudaSuccess;
}

namespace {

using gsx::fcompress;
using gsx::fnode;
using gsx::V16;

constexpr int kMaxWarps = 32;

template <class T, int DIM, int A>
__global__ void __launch_bounds__(512) coarse_gs_kernel(Geom g, LevelDev<T> t, CellData cd,
                                                        Schedule sc, int ndir,
                                                        const int* __restrict__ dir_begin,
                                                        const int* __restrict__ dir_end,
                                                        int sweeps, const T* __restrict__ f,
                                                        T* __restrict__ psi, T* __restrict__ mom) {
  constexpr int S = 1 << DIM;
  constexpr int SA = S * A;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ T delta_s[kMaxWarps][SA];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int wpc = blockDim.x >> 5;
  const int gw = (int)cluster.block_rank() * wpc + wib;
  const int W = (int)cluster.num_blocks() * wpc;
  const int nm = t.nmom;
  const int nadof = g.nadof;
  const bool act = lane < SA;
  const int l = act ? lane / A : 0;
  const int m = act ? lane % A : 0;
  const int stride[3] = {1, g.nx, g.nx * g.ny};
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int d = 0; d < ndir; ++d) {
      int neg[3];
      if (DIM == 2) {
        neg[0] = (d >> 1) & 1; neg[1] = d & 1; neg[2] = 0;
      } else {
        neg[0] = (d >> 2) & 1; neg[1] = (d >> 1) & 1; neg[2] = d & 1;
      }
      const int qb = dir_begin[d], qe = dir_end[d];
      for (int w = 0; w < sc.nlev; ++w) {
        const int beg = sc.level_off[w];
        const int cnt = sc.level_off[w + 1] - beg;
        for (int k = gw; k < cnt; k += W) {
          const int packed = sc.cells[beg + k];
          const int jj[3] = {packed & 2047, (packed >> 11) & 2047, packed >> 22};
          const int ix = neg[0] ? g.nx - 1 - jj[0] : jj[0];
          const int iy = neg[1] ? g.ny - 1 - jj[1] : jj[1];
          const int iz = neg[2] ? g.nz - 1 - jj[2] : jj[2];
          const int c = ix + g.nx * (iy + g.ny * iz);
          T* Phi = mom + (long long)c * S * nm;
          const int mat = cd.mat[c];
          const T sig_s = (T)cd.sigma_s[c];
          const int sh = cd.fid ? cd.fid[c] : 0;  // the cell's moment shape
          const T* xfs = t.XFt + (size_t)sh * nm * nadof;
          const T* sqs = t.Sqq + (size_t)sh * g.P * A * A;
          for (int q = qb; q < qe; ++q) {
            const long long off = ((long long)c * S + l) * nadof + q * A + m;
            T rhs = act ? f[off] : T(0);
            const T old = act ? __ldcg(psi + off) : T(0);
            if (act) {
              // upwind term of this (l, m) entry
#pragma unroll
              for (int xi = 0; xi < DIM; ++xi) {
                if (jj[xi] == 0) continue;
                const int own = neg[xi];
                if (((l >> xi) & 1) != own) continue;
                const int cn = c + (own ? stride[xi] : -stride[xi]);
                const T nsgn = own ? T(1) : T(-1);
                const T* An = t.Aax + ((size_t)q * 3 + xi) * A * A + m * A;
                const int jp = fcompress(l, xi);
                const T* pn = psi + (long long)cn * S * nadof + q * A;
                T acc = T(0);
#pragma unroll
                for (int j = 0; j < S / 2; ++j) {
                  const int i = fnode(j, xi, 1 - own);
                  T sacc = T(0);
#pragma unroll
                  for (int dd = 0; dd < A; ++dd) sacc += An[dd] * __ldcg(pn + (long long)i * nadof + dd);
                  acc += T(g.facemass[xi][jp][j]) * sacc;
                }
                rhs -= nsgn * acc;
              }
            }
            // G[l][m] = (X_q F Phi_c)[m][l] - (S_qq x_old)[l][m]
            T G = T(0);
            if (act) {
              const T* xf = xfs;  // [nm][nadof]
              for (int kk = 0; kk < nm; ++kk) G += xf[(long long)kk * nadof + q * A + m] * __ldcg(Phi + l * nm + kk);
            }
            const T* Sq = sqs + (size_t)q * A * A;
#pragma unroll
            for (int dd = 0; dd < A; ++dd) {
              const T od = __shfl_sync(0xffffffffu, old, l * A + dd);
              G -= act ? Sq[m * A + dd] * od : T(0);
            }
            // Q[l][m] = sigma_s sum_i N[l][i] G[i][m]
            T Q = T(0);
#pragma unroll
            for (int i = 0; i < S; ++i) {
              const T gi = __shfl_sync(0xffffffffu, G, i * A + m);
              Q += (T)g.Nmass[l * S + i] * gi;
            }
            rhs += sig_s * Q;
            // x = Ginv rhs
            const T* Gi = t.Ginv + ((size_t)mat * g.P + q) * SA * SA + (act ? lane : 0) * SA;
            T x = T(0);
#pragma unroll
            for (int j = 0; j < SA; ++j) {
              const T rj = __shfl_sync(0xffffffffu, rhs, j);
              x += Gi[j] * rj;
            }
            if (act) {
              psi[off] = x;
              delta_s[wib][lane] = x - old;
            }
            __syncwarp();
            // Phi_c[i][k] += sum_d X[q*A+d][k] delta[i][d]
            for (int e = lane; e < S * nm; e += 32) {
              const int i = e / nm, kk = e - (e / nm) * nm;
              T acc = T(0);
#pragma unroll
              for (int dd = 0; dd < A; ++dd)
                acc += t.X[(long long)(q * A + dd) * nm + kk] * delta_s[wib][i * A + dd];
              Phi[i * nm + kk] = __ldcg(Phi + i * nm + kk) + acc;
            }
            __syncwarp();
          }
        }
        cluster.sync();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Direction-blocked form of the same Gauss-Seidel sweep.  For the patches Q_d
// of sweep direction d in one cell, visiting them in index order with the
// latest values is one forward block substitution with the block lower
// triangle of the cell-direction matrix:
//   (D_d - sigma_s N (x) S_dd^{L+D}) x_d^new
//       = f_d - up_d + sigma_s N (x) (S_{d,all} x^cur - S_dd^{L+D} x_d^old),
// where D_d = blockdiag_q(K0_q + sigma_t B_q), S_dd^{L+D} keeps the blocks
// S_qp with p <= q, and S_{d,all} x^cur = X_d F Phi_c (moment form).  The
// inverse of the left-hand matrix, Tinv[mat][d] (E x E, E = s * |Q_d| * a,
// stored transposed), is precomputed, so the |Q_d| sequential patch solves
// become one matrix-vector product -- the same result up to rounding.
// Each warp owns one cell at a time and keeps its data in shared memory.
template <class T, int DIM, int A>
__global__ void __launch_bounds__(512) coarse_gs_block_kernel(
    Geom g, LevelDev<T> t, CellData cd, Schedule sc, int ndir, const int* __restrict__ dir_begin,
    const int* __restrict__ dir_end, int sweeps, const T* __restrict__ f, T* __restrict__ psi,
    T* __restrict__ mom, const T* __restrict__ TinvT, const T* __restrict__ SLD, int Emax,
    int Jmax) {
  constexpr int S = 1 << DIM;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int wpc = blockDim.x >> 5;
  const int gw = (int)cluster.block_rank() * wpc + wib;
  const int W = (int)cluster.num_blocks() * wpc;
  const int nm = t.nmom;
  const int nadof = g.nadof;
  // per-warp workspace: rhs[Emax], xold[Emax], buf[Emax], phi[S*nm]
  T* ws = reinterpret_cast<T*>(smem_raw) + (size_t)wib * (3 * Emax + S * nm);
  T* rhs = ws;
  T* xold = ws + Emax;
  T* buf = ws + 2 * Emax;
  T* phs = ws + 3 * Emax;
  const int stride[3] = {1, g.nx, g.nx * g.ny};
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int d = 0; d < ndir; ++d) {
      int neg[3];
      if (DIM == 2) {
        neg[0] = (d >> 1) & 1; neg[1] = d & 1; neg[2] = 0;
      } else {
        neg[0] = (d >> 2) & 1; neg[1] = (d >> 1) & 1; neg[2] = d & 1;
      }
      const int qb = dir_begin[d];
      const int J = (dir_end[d] - qb) * A;
      const int E = S * J;
      const T* SLDd = SLD + (size_t)d * Jmax * Jmax;
      for (int w = 0; w < sc.nlev; ++w) {
        const int beg = sc.level_off[w];
        const int cnt = sc.level_off[w + 1] - beg;
        for (int k = gw; k < cnt; k += W) {
          const int packed = sc.cells[beg + k];
          const int jj[3] = {packed & 2047, (packed >> 11) & 2047, packed >> 22};
          const int ix = neg[0] ? g.nx - 1 - jj[0] : jj[0];
          const int iy = neg[1] ? g.ny - 1 - jj[1] : jj[1];
          const int iz = neg[2] ? g.nz - 1 - jj[2] : jj[2];
          const int c = ix + g.nx * (iy + g.ny * iz);
          const int mat = cd.mat[c];
          const T sig_s = (T)cd.sigma_s[c];
          T* Phi = mom + (long long)c * S * nm;
          // 1. loads: f - upwind, old values, cell moments
          for (int e = lane; e < E; e += 32) {
            const int l = e / J, j = e - (e / J) * J;
            const int q = qb + j / A, m = j % A;
            const long long gi = ((long long)c * S + l) * nadof + qb * A + j;
            T r = f[gi];
            xold[e] = __ldcg(psi + gi);
#pragma unroll
            for (int xi = 0; xi < DIM; ++xi) {
              if (jj[xi] == 0) continue;
              const int own = neg[xi];
              if (((l >> xi) & 1) != own) continue;
              const int cn = c + (own ? stride[xi] : -stride[xi]);
              const T nsgn = own ? T(1) : T(-1);
              const T* An = t.Aax + ((size_t)q * 3 + xi) * A * A + m * A;
              const int jp = fcompress(l, xi);
              const T* pn = psi + (long long)cn * S * nadof + q * A;
              T acc = T(0);
#pragma unroll
              for (int j2 = 0; j2 < S / 2; ++j2) {
                const int i = fnode(j2, xi, 1 - own);
                T sacc = T(0);
#pragma unroll
                for (int dd = 0; dd < A; ++dd) sacc += An[dd] * __ldcg(pn + (long long)i * nadof + dd);
                acc += T(g.facemass[xi][jp][j2]) * sacc;
              }
              r -= nsgn * acc;
            }
            rhs[e] = r;
          }
          for (int e = lane; e < S * nm; e += 32) phs[e] = __ldcg(Phi + e);
          __syncwarp();
          // 2. buf = X_d F Phi - S_dd^{L+D} x_old   (entry (l, j))
          for (int e = lane; e < E; e += 32) {
            const int l = e / J, j = e - (e / J) * J;
            T acc = T(0);
            const T* xf = t.XFt + qb * A + j;
            for (int kk = 0; kk < nm; ++kk) acc += xf[(long long)kk * nadof] * phs[l * nm + kk];
            const T* sl = SLDd + (size_t)j * Jmax;
            const T* xo = xold + l * J;
            for (int j2 = 0; j2 < J; ++j2) acc -= sl[j2] * xo[j2];
            buf[e] = acc;
          }
          __syncwarp();
          // 3. rhs += sigma_s N (x) buf
          for (int e = lane; e < E; e += 32) {
            const int l = e / J, j = e - (e / J) * J;
            T acc = T(0);
#pragma unroll
            for (int i = 0; i < S; ++i) acc += (T)g.Nmass[l * S + i] * buf[i * J + j];
            rhs[e] += sig_s * acc;
          }
          __syncwarp();
          // 4. x_new = Tinv rhs  (Tinv stored transposed: TinvT[col][row])
          const T* Tm = TinvT + ((size_t)mat * ndir + d) * Emax * Emax;
          for (int r = lane; r < E; r += 32) {
            T acc = T(0);
            for (int cc = 0; cc < E; ++cc) acc += Tm[(size_t)cc * Emax + r] * rhs[cc];
            buf[r] = acc;
          }
          __syncwarp();
          // 5. store, delta
          for (int e = lane; e < E; e += 32) {
            const int l = e / J, j = e - (e / J) * J;
            const long long gi = ((long long)c * S + l) * nadof + qb * A + j;
            psi[gi] = buf[e];
            xold[e] = buf[e] - xold[e];
          }
          __syncwarp();
          // 6. Phi_c += X_d^T delta
          for (int e = lane; e < S * nm; e += 32) {
            const int l = e / nm, kk = e - (e / nm) * nm;
            T acc = T(0);
            const T* xr = t.X + (long long)(qb * A) * nm + kk;
            const T* dl = xold + l * J;
            for (int j = 0; j < J; ++j) acc += xr[(long long)j * nm] * dl[j];
            Phi[e] = phs[e] + acc;
          }
          __syncwarp();
        }
        cluster.sync();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Thread-group form of the direction-blocked sweep: one group of GT threads
// (GT >= E, a multiple of 32) per cell, one thread per block entry, and the
// direction's tables -- the block inverses of every material, X_d, diag(f)X_d^T
// and S_dd^{L+D} -- staged in shared memory once per direction.  Groups of one
// thread block synchronise with named barriers; wavefront levels with the
// cluster barrier.
__device__ __forceinline__ void group_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident): a
// counter and a generation word in global memory; the last block to arrive
// resets the counter and advances the generation.  The wait is bounded (2 s);
// on timeout the block records code 4 in `err` and continues.
__device__ __forceinline__ void grid_barrier(unsigned* bar, unsigned nblocks, unsigned& gen,
                                             int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == nblocks) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicExch(bar + 1, gen + 1u);
    } else {
      const unsigned long long t0 = gsx::now_ns();
      unsigned it = 0;
      while (*vgen == gen) {
        if ((++it & 255u) == 0 && gsx::now_ns() - t0 > 2000000000ULL) {
          atomicExch(err, 4);
          break;
        }
      }
    }
    __threadfence();
  }
  gen += 1u;
  __syncthreads();
}

template <class T, int DIM, int A, bool VEC, bool GRID>
__global__ void __launch_bounds__(768) coarse_gs_group_kernel(
    Geom g, LevelDev<T> t, CellData cd, Schedule sc, int ndir, const int* __restrict__ dir_begin,
    const int* __restrict__ dir_end, int sweeps, const T* __restrict__ f, T* __restrict__ psi,
    T* __restrict__ mom, const T* __restrict__ TinvT, const T* __restrict__ SLD, int Emax,
    int Jmax, int nmat, int GT, unsigned* __restrict__ gbar, int* __restrict__ err) {
  constexpr int S = 1 << DIM;
  constexpr int HS = S / 2;
  constexpr int VW = 16 / (int)sizeof(T);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nm = t.nmom;
  const int nadof = g.nadof;
  const int ngroups = blockDim.x / GT;
  const int gi = threadIdx.x / GT;
  const int r = threadIdx.x - gi * GT;
  int rank, nblocks;
  if constexpr (GRID) {
    rank = blockIdx.x;
    nblocks = gridDim.x;
  } else {
    cg::cluster_group cl = cg::this_cluster();
    rank = (int)cl.block_rank();
    nblocks = (int)cl.num_blocks();
  }
  const int gg = rank * ngroups + gi;
  const int G = nblocks * ngroups;
  unsigned gen = 0;  // grid barrier generation seen by this block
  auto level_barrier = [&]() {
    if constexpr (GRID) {
      grid_barrier(gbar, (unsigned)nblocks, gen, err);
    } else {
      cg::this_cluster().sync();
    }
  };
  const int Ep = gsx::pad16<T>(Emax), NMp = gsx::pad16<T>(nm), Jp = gsx::pad16<T>(Jmax);
  // shared layout (every sub-array starts on a 16-byte boundary)
  T* Tin = reinterpret_cast<T*>(smem_raw);                           // [nmat][Emax][Ep]
  T* XFr = Tin + gsx::round16((size_t)nmat * Emax * Ep, sizeof(T));    // [Jmax][NMp]
  T* Xk = XFr + gsx::round16((size_t)Jmax * NMp, sizeof(T));           // [nm][Jp]
  T* SLr = Xk + gsx::round16((size_t)nm * Jp, sizeof(T));              // [Jmax][Jp]
  T* Ns = SLr + gsx::round16((size_t)Jmax * Jp, sizeof(T));            // [S*S]
  const size_t per_group = gsx::round16(3 * (size_t)Emax, sizeof(T)) +
                           gsx::round16((size_t)S * NMp, sizeof(T)) +
                           gsx::round16((size_t)DIM * HS * Jmax, sizeof(T));
  T* ws = Ns + gsx::round16(S * S, sizeof(T)) + (size_t)gi * per_group;
  T* rhs = ws;
  T* xold = ws + Emax;
  T* buf = ws + 2 * Emax;
  T* phs = ws + gsx::round16(3 * (size_t)Emax, sizeof(T));            // [S][NMp]
  T* upw = phs + gsx::round16((size_t)S * NMp, sizeof(T));             // [DIM][HS][J]
  const int bid = 1 + gi;  // named barrier of this group (0 is __syncthreads)
  for (int i = threadIdx.x; i < S * S; i += blockDim.x) Ns[i] = (T)g.Nmass[i];
  for (int i = r; i < S * NMp; i += GT) phs[i] = T(0);  // padding stays zero
  constexpr int MAXE = 2;  // E <= 2 GT
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int d = 0; d < ndir; ++d) {
      int n0, n1, n2;
      if (DIM == 2) {
        n0 = (d >> 1) & 1; n1 = d & 1; n2 = 0;
      } else {
        n0 = (d >> 2) & 1; n1 = (d >> 1) & 1; n2 = d & 1;
      }
      const int qb = dir_begin[d];
      const int J = (dir_end[d] - qb) * A;
      const int E = S * J;
      // stage this direction's tables (the previous level ended with a cluster barrier)
      for (int mt = 0; mt < nmat; ++mt) {
        const T* src = TinvT + ((size_t)mt * ndir + d) * Emax * Emax;  // [col][row]
        T* dst = Tin + (size_t)mt * Emax * Ep;                           // [row][col]
        for (int i = threadIdx.x; i < Emax * Emax; i += blockDim.x) {
          const int col = i / Emax, row = i - col * Emax;
          dst[(size_t)row * Ep + col] = (row < E && col < E) ? src[i] : T(0);
        }
      }
      for (int i = threadIdx.x; i < Jmax * NMp; i += blockDim.x) {
        const int j = i / NMp, kk = i - j * NMp;
        XFr[i] = (j < J && kk < nm) ? t.XFt[(long long)kk * nadof + qb * A + j] : T(0);
      }
      for (int i = threadIdx.x; i < nm * Jp; i += blockDim.x) {
        const int kk = i / Jp, j = i - kk * Jp;
        Xk[i] = j < J ? t.X[(long long)(qb * A + j) * nm + kk] : T(0);
      }
      for (int i = threadIdx.x; i < Jmax * Jp; i += blockDim.x) {
        const int j = i / Jp, j2 = i - j * Jp;
        SLr[i] = (j < J && j2 < J) ? SLD[((size_t)d * Jmax + j) * Jmax + j2] : T(0);
      }
      __syncthreads();
      // rotated coordinates of the k-th cell of wavefront level w (in 2D by
      // arithmetic: cells of a level are ordered by increasing row)
      auto rot_of = [&](int w, int k, int& j0, int& j1, int& j2c) {
        if (DIM == 2) {
          j1 = max(0, w - (g.nx - 1)) + k;
          j0 = w - j1;
          j2c = 0;
        } else {
          const int packed = sc.cells[sc.level_off[w] + k];
          j0 = packed & 2047; j1 = (packed >> 11) & 2047; j2c = packed >> 22;
        }
      };
      auto count_of = [&](int w) {
        if (DIM == 2) return min(w, g.ny - 1) - max(0, w - (g.nx - 1)) + 1;
        return sc.level_off[w + 1] - sc.level_off[w];
      };
      auto cell_of = [&](int w, int k) {
        int j0, j1, j2c;
        rot_of(w, k, j0, j1, j2c);
        const int ix = n0 ? g.nx - 1 - j0 : j0;
        const int iy = n1 ? g.ny - 1 - j1 : j1;
        const int iz = n2 ? g.nz - 1 - j2c : j2c;
        return ix + g.nx * (iy + g.ny * iz);
      };
      // prefetch registers for the group's cell at the next level
      T pf[MAXE], px[MAXE], pm[4];
      auto prefetch = [&](int w, int kk) {
        const int cnt = count_of(w);
        if (kk >= cnt) return;
        const int c = cell_of(w, kk);
#pragma unroll
        for (int u = 0; u < MAXE; ++u) {
          const int e = r + u * GT;
          if (e < E) {
            const int l = e / J, j = e - l * J;
            const long long gix = ((long long)c * S + l) * nadof + qb * A + j;
            pf[u] = f[gix];
            px[u] = __ldcg(psi + gix);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = r + u * GT;
          if (e < S * nm) pm[u] = __ldcg(mom + (long long)c * S * nm + e);
        }
      };
      if (sc.nlev > 0) prefetch(0, gg);
      for (int w = 0; w < sc.nlev; ++w) {
        const int cnt = count_of(w);
        bool prefetched = false;
       for (int k = gg; k < cnt; k += G) {
        const bool have = true;
        if (k == gg) {
          // the group's first cell of this level was prefetched one level ago
#pragma unroll
          for (int u = 0; u < MAXE; ++u) {
            const int e = r + u * GT;
            if (e < E) {
              rhs[e] = pf[u];
              xold[e] = px[u];
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int e = r + u * GT;
            if (e < S * nm) {
              const int l = e / nm;
              phs[l * NMp + (e - l * nm)] = pm[u];
            }
          }
        } else {
          // further cells of this group on the same level: load directly
          const int c2 = cell_of(w, k);
          for (int e = r; e < E; e += GT) {
            const int l = e / J, j = e - l * J;
            const long long gix = ((long long)c2 * S + l) * nadof + qb * A + j;
            rhs[e] = f[gix];
            xold[e] = __ldcg(psi + gix);
          }
          for (int e = r; e < S * nm; e += GT) {
            const int l = e / nm;
            phs[l * NMp + (e - l * nm)] = __ldcg(mom + (long long)c2 * S * nm + e);
          }
        }
        int c = 0, jj0 = 0, jj1 = 0, jj2 = 0;
        if (have) {
          rot_of(w, k, jj0, jj1, jj2);
          c = cell_of(w, k);
          for (int e = r; e < DIM * HS * J; e += GT) {
            const int xi = e / (HS * J);
            const int rem = e - xi * HS * J;
            const int jn = rem / J, j = rem - jn * J;
            const int jx = xi == 0 ? jj0 : (xi == 1 ? jj1 : jj2);
            T v = T(0);
            if (jx > 0) {
              const int own = xi == 0 ? n0 : (xi == 1 ? n1 : n2);
              const int strd = xi == 0 ? 1 : (xi == 1 ? g.nx : g.nx * g.ny);
              const int cn = c + (own ? strd : -strd);
              const int i = fnode(jn, xi, 1 - own);
              v = __ldcg(psi + ((long long)cn * S + i) * nadof + qb * A + j);
            }
            upw[e] = v;
          }
        }
        if (k == gg && w + 1 < sc.nlev) {
          prefetch(w + 1, gg);  // the registers of this level's first cell are in shared memory
          prefetched = true;
        }
        if (have) {
          const int mat = cd.mat[c];
          const T sig_s = (T)cd.sigma_s[c];
          T* Phi = mom + (long long)c * S * nm;
          group_bar(bid, GT);
          // 1-2. rhs = f - upwind;  buf = X_d F Phi - S_dd^{L+D} x_old
          for (int e = r; e < E; e += GT) {
            const int l = e / J, j = e - l * J;
            const int q = qb + j / A, m = j % A;
            T val = rhs[e];
#pragma unroll
            for (int xi = 0; xi < DIM; ++xi) {
              const int jx = xi == 0 ? jj0 : (xi == 1 ? jj1 : jj2);
              const int own = xi == 0 ? n0 : (xi == 1 ? n1 : n2);
              if (jx == 0 || ((l >> xi) & 1) != own) continue;
              const T* An = t.Aax + ((size_t)q * 3 + xi) * A * A + m * A;
              const int jp = fcompress(l, xi);
              const int jb = (j / A) * A;
              T acc = T(0);
#pragma unroll
              for (int jn = 0; jn < HS; ++jn) {
                const T* nv = upw + (xi * HS + jn) * J + jb;
                T sacc = T(0);
#pragma unroll
                for (int dd = 0; dd < A; ++dd) sacc += An[dd] * nv[dd];
                acc += T(g.facemass[xi][jp][jn]) * sacc;
              }
              val -= (own ? T(1) : T(-1)) * acc;
            }
            rhs[e] = val;
            T a0 = T(0), a1 = T(0);
            if constexpr (VEC) {
              const T* xr = XFr + j * NMp;
              const T* ph = phs + l * NMp;
              for (int kk = 0; kk < NMp; kk += VW) a0 += V16<T>::dot(xr + kk, ph + kk);
              const T* sl = SLr + j * Jp;
              const T* xo = xold + l * J;
              for (int j3 = 0; j3 < J; j3 += VW) a1 -= V16<T>::dot(sl + j3, xo + j3);
            } else {
              const T* ph = phs + l * NMp;
              for (int kk = 0; kk < nm; ++kk) a0 += XFr[j * NMp + kk] * ph[kk];
              const T* xo = xold + l * J;
              for (int j3 = 0; j3 < J; ++j3) a1 -= SLr[j * Jp + j3] * xo[j3];
            }
            buf[e] = a0 + a1;
          }
          group_bar(bid, GT);
          // 3. rhs += sigma_s N (x) buf
          for (int e = r; e < E; e += GT) {
            const int l = e / J, j = e - l * J;
            T acc = T(0);
#pragma unroll
            for (int i = 0; i < S; ++i) acc += Ns[l * S + i] * buf[i * J + j];
            rhs[e] += sig_s * acc;
          }
          group_bar(bid, GT);
          // 4. x_new = Tinv rhs
          const T* Tm = Tin + (size_t)mat * Emax * Ep;
          for (int rr = r; rr < E; rr += GT) {
            T a0 = T(0), a1 = T(0);
            const T* row = Tm + (size_t)rr * Ep;
            if constexpr (VEC) {
              int cc = 0;
              for (; cc + 2 * VW <= E; cc += 2 * VW) {
                a0 += V16<T>::dot(row + cc, rhs + cc);
                a1 += V16<T>::dot(row + cc + VW, rhs + cc + VW);
              }
              for (; cc < E; cc += VW) a0 += V16<T>::dot(row + cc, rhs + cc);
            } else {
              for (int cc = 0; cc < E; ++cc) a0 += row[cc] * rhs[cc];
            }
            const T xn = a0 + a1;
            const int l = rr / J, j = rr - l * J;
            psi[((long long)c * S + l) * nadof + qb * A + j] = xn;
            buf[rr] = xn - xold[rr];
          }
          group_bar(bid, GT);
          // 5. Phi_c += X_d^T delta
          for (int e = r; e < S * nm; e += GT) {
            const int l = e / nm, kk = e - l * nm;
            T a0 = T(0);
            const T* xr = Xk + kk * Jp;
            const T* dl = buf + l * J;
            if constexpr (VEC) {
              for (int j = 0; j < J; j += VW) a0 += V16<T>::dot(xr + j, dl + j);
            } else {
              for (int j = 0; j < J; ++j) a0 += xr[j] * dl[j];
            }
            Phi[e] = phs[l * NMp + kk] + a0;
          }
          group_bar(bid, GT);  // the workspace is reused by the next cell
        }
       }
        if (!prefetched && w + 1 < sc.nlev) prefetch(w + 1, gg);
        level_barrier();
      }
    }
  }
}

template <class T>
size_t gs_group_tables_bytes(int nmat, int Emax, int Jmax, int nm, int s) {
  const int Ep = gsx::pad16<T>(Emax), NMp = gsx::pad16<T>(nm), Jp = gsx::pad16<T>(Jmax);
  return (gsx::round16((size_t)nmat * Emax * Ep, sizeof(T)) + gsx::round16((size_t)Jmax * NMp, sizeof(T)) +
          gsx::round16((size_t)nm * Jp, sizeof(T)) + gsx::round16((size_t)Jmax * Jp, sizeof(T)) +
          gsx::round16((size_t)s * s, sizeof(T))) * sizeof(T);
}
template <class T>
size_t gs_group_bytes(int Emax, int Jmax, int nm, int s, int dim) {
  const int NMp = gsx::pad16<T>(nm);
  return (gsx::round16(3 * (size_t)Emax, sizeof(T)) + gsx::round16((size_t)s * NMp, sizeof(T)) +
          gsx::round16((size_t)dim * (s / 2) * Jmax, sizeof(T))) * sizeof(T);
}

template <class T, int DIM, int A, bool VEC>
cudaError_t launch_gs_grid_impl(int nblocks, int ngroups, int GT, size_t smem, const Geom& g,
                                const LevelDev<T>& t, const CellData& cd, const Schedule& sc,
                                int ndir, const int* db, const int* de, int sweeps, const T* f,
                                T* phi, T* mom, const T* TinvT, const T* SLD, int Emax, int Jmax,
                                int nmat, unsigned* gbar, int* err, cudaStream_t st) {
  auto kern = coarse_gs_group_kernel<T, DIM, A, VEC, true>;
  cudaError_t e = allow_max_smem(kern);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, ngroups * GT, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (per_sm < 1 || nblocks > per_sm * nsm) return cudaErrorCooperativeLaunchTooLarge;
  e = cudaMemsetAsync(gbar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&g, (void*)&t, (void*)&cd, (void*)&sc, (void*)&ndir, (void*)&db,
                  (void*)&de, (void*)&sweeps, (void*)&f, (void*)&phi, (void*)&mom,
                  (void*)&TinvT, (void*)&SLD, (void*)&Emax, (void*)&Jmax, (void*)&nmat,
                  (void*)&GT, (void*)&gbar, (void*)&err};
  return cudaLaunchCooperativeKernel((void*)kern, dim3(nblocks), dim3(ngroups * GT), args, smem,
                                     st);
}

template <class T, int DIM, int A, bool VEC>
cudaError_t launch_gs_group_impl(int cl, int ngroups, int GT, size_t smem, const Geom& g,
                                 const LevelDev<T>& t, const CellData& cd, const Schedule& sc,
                                 int ndir, const int* db, const int* de, int sweeps, const T* f,
                                 T* phi, T* mom, const T* TinvT, const T* SLD, int Emax, int Jmax,
                                 int nmat, cudaStream_t st) {
  auto kern = coarse_gs_group_kernel<T, DIM, A, VEC, false>;
  cudaError_t e = allow_max_smem(kern);
  if (e != cudaSuccess) return e;
  if (cl > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(ngroups * GT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (nclusters < 1) return cudaErrorLaunchOutOfResources;
  unsigned* nobar = nullptr;
  int* noerr = nullptr;
  return cudaLaunchKernelEx(&cfg, kern, g, t, cd, sc, ndir, db, de, sweeps, f, phi, mom, TinvT,
                            SLD, Emax, Jmax, nmat, GT, nobar, noerr);
}

template <class T, int DIM, int A>
cudaError_t launch_gs_block_impl(int cl, int wpc, const Geom& g, const LevelDev<T>& t,
                                 const CellData& cd, const Schedule& sc, int ndir, const int* db,
                                 const int* de, int sweeps, const T* f, T* phi, T* mom,
                                 const T* TinvT, const T* SLD, int Emax, int Jmax,
                                 cudaStream_t st) {
  auto kern = coarse_gs_block_kernel<T, DIM, A>;
  const size_t smem = (size_t)wpc * (3 * Emax + (1 << DIM) * t.nmom) * sizeof(T);
  cudaError_t e = allow_max_smem(kern);
  if (e != cudaSuccess) return e;
  if (cl > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(32 * wpc);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (nclusters < 1) return cudaErrorLaunchOutOfResources;
  return cudaLaunchKernelEx(&cfg, kern, g, t, cd, sc, ndir, db, de, sweeps, f, phi, mom, TinvT,
                            SLD, Emax, Jmax);
}

template <class T, int DIM, int A>
cudaError_t launch_gs_impl(int cl, const Geom& g, const LevelDev<T>& t, const CellData& cd,
                           const Schedule& sc, int ndir, const int* db, const int* de,
                           int sweeps, const T* f, T* phi, T* mom, cudaStream_t st) {
  auto kern = coarse_gs_kernel<T, DIM, A>;
  if (cl > 8) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // only launch a cluster shape the device can co-schedule
  int nclusters = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (nclusters < 1) return cudaErrorLaunchOutOfResources;
  return cudaLaunchKernelEx(&cfg, kern, g, t, cd, sc, ndir, db, de, sweeps, f, phi, mom);
}

}  // namespace

template <class T>
void launch_coarse_gs(const Geom& g, const LevelDev<T>& t, const CellData& cd,
                      const Schedule& sc, int ndir, const int* dir_begin, const int* dir_end,
                      int sweeps, const T* f, T* phi, T* moments, int* status,
                      cudaStream_t st) {
  // the largest cluster the device accepts: 16 CTAs (non-portable), else 8, else 1
  const int sizes[3] = {16, 8, 1};
  for (int cl : sizes) {
    cudaError_t e;
    if (g.dim == 2 && g.a == 3)
      e = launch_gs_impl<T, 2, 3>(cl, g, t, cd, sc, ndir, dir_begin, dir_end, sweeps, f, phi, moments, st);
    else if (g.dim == 2)
      e = launch_gs_impl<T, 2, 1>(cl, g, t, cd, sc, ndir, dir_begin, dir_end, sweeps, f, phi, moments, st);
    else if (g.a == 3)
      e = launch_gs_impl<T, 3, 3>(cl, g, t, cd, sc, ndir, dir_begin, dir_end, sweeps, f, phi, moments, st);
    else
      e = launch_gs_impl<T, 3, 1>(cl, g, t, cd, sc, ndir, dir_begin, dir_end, sweeps, f, phi, moments, st);
    if (e == cudaSuccess) {
      note_launch();
      if (status) *status = cl;
      return;
    }
    cudaGetLastError();  // clear and try a smaller cluster
  }
  if (status) *status = 0;
}

template <class T>
void launch_coarse_gs_block(const Geom& g, const LevelDev<T>& t, const CellData& cd,
                            const Schedule& sc, int ndir, const int* dir_begin,
                            const int* dir_end, int sweeps, const T* f, T* phi, T* moments,
                            const T* TinvT, const T* SLD, int Emax, int Jmax, int nmat,
                            int variant, int vec_ok, int max_level_cells, int grid_blocks,
                            unsigned* gbar, int* err, int* status, cudaStream_t st) {
  int sizes[3] = {16, 8, 1};
  if (grid_blocks < 0) {  // negative: a fixed cluster size for the cluster kernels
    sizes[0] = sizes[1] = sizes[2] = -grid_blocks;
    grid_blocks = 0;
  }
  // thread-group kernel: tables of all materials in shared memory
  {
    const int GT = ((Emax + 31) / 32) * 32;
    const size_t tables = gs_group_tables_bytes<T>(nmat, Emax, Jmax, t.nmom, g.s);
    const size_t per_group = gs_group_bytes<T>(Emax, Jmax, t.nmom, g.s, g.dim);
    int ngroups = std::min(15, 768 / GT);
    while (ngroups > 1 && tables + ngroups * per_group > 220 * 1024) --ngroups;
    // the vector path needs every direction's J to be a multiple of 16 bytes
    const bool vec = (sizeof(T) == 4 ? (vec_ok & 1) : (vec_ok & 2)) != 0;
    if (variant == 4 && GT <= 128 && Emax <= 2 * GT && g.s * t.nmom <= 4 * GT &&
        tables + per_group <= 220 * 1024 && gbar) {
      // whole-GPU form: one group per block, one block per cell of the widest level
      const size_t smem = tables + per_group;
      const int nb = std::min(std::max(1, max_level_cells), grid_blocks > 0 ? grid_blocks : 148);
      cudaError_t e;
#define AMGT_GS_GRID(DIM_, A_)                                                                   \
  (vec ? launch_gs_grid_impl<T, DIM_, A_, true>(nb, 1, GT, smem, g, t, cd, sc, ndir, dir_begin,  \
                                                 dir_end, sweeps, f, phi, moments, TinvT, SLD,   \
                                                 Emax, Jmax, nmat, gbar, err, st)                \
       : launch_gs_grid_impl<T, DIM_, A_, false>(nb, 1, GT, smem, g, t, cd, sc, ndir, dir_begin, \
                                                  dir_end, sweeps, f, phi, moments, TinvT, SLD,  \
                                                  Emax, Jmax, nmat, gbar, err, st))
      if (g.dim == 2 && g.a == 3) e = AMGT_GS_GRID(2, 3);
      else if (g.dim == 2) e = AMGT_GS_GRID(2, 1);
      else if (g.a == 3) e = AMGT_GS_GRID(3, 3);
      else e = AMGT_GS_GRID(3, 1);
#undef AMGT_GS_GRID
      if (e == cudaSuccess) {
        note_launch();
        if (status) *status = 200;
        return;
      }
      cudaGetLastError();
    }
    if (variant != 2 && GT <= 128 && Emax <= 2 * GT && g.s * t.nmom <= 4 * GT &&
        tables + ngroups * per_group <= 220 * 1024) {
      const size_t smem = tables + ngroups * per_group;
      for (int cl : sizes) {
        cudaError_t e;
#define AMGT_GS_LAUNCH(DIM_, A_)                                                                 \
  (vec ? launch_gs_group_impl<T, DIM_, A_, true>(cl, ngroups, GT, smem, g, t, cd, sc, ndir,      \
                                                  dir_begin, dir_end, sweeps, f, phi, moments,   \
                                                  TinvT, SLD, Emax, Jmax, nmat, st)              \
       : launch_gs_group_impl<T, DIM_, A_, false>(cl, ngroups, GT, smem, g, t, cd, sc, ndir,     \
                                                   dir_begin, dir_end, sweeps, f, phi, moments,  \
                                                   TinvT, SLD, Emax, Jmax, nmat, st))
        if (g.dim == 2 && g.a == 3) e = AMGT_GS_LAUNCH(2, 3);
        else if (g.dim == 2) e = AMGT_GS_LAUNCH(2, 1);
        else if (g.a == 3) e = AMGT_GS_LAUNCH(3, 3);
        else e = AMGT_GS_LAUNCH(3, 1);
#undef AMGT_GS_LAUNCH
        if (e == cudaSuccess) {
          note_launch();
          if (status) *status = 100 + cl;
          return;
        }
        cudaGetLastError();
      }
    }
  }
  const size_t per_warp = (size_t)(3 * Emax + g.s * t.nmom) * sizeof(T);
  int wpc = 16;
  while (wpc > 1 && per_warp * wpc > 200 * 1024) wpc /= 2;
  for (int cl : sizes) {
    cudaError_t e;
    if (g.dim == 2 && g.a == 3)
      e = launch_gs_block_impl<T, 2, 3>(cl, wpc, g, t, cd, sc, ndir, dir_begin, dir_end, sweeps, f, phi, moments, TinvT, SLD, Emax, Jmax, st);
    else if (g.dim == 2)
      e = launch_gs_block_impl<T, 2, 1>(cl, wpc, g, t, cd, sc, ndir, dir_begin, dir_end, sweeps, f, phi, moments, TinvT, SLD, Emax, Jmax, st);
    else if (g.a == 3)
      e = launch_gs_block_impl<T, 3, 3>(cl, wpc, g, t, cd, sc, ndir, dir_begin, dir_end, sweeps, f, phi, moments, TinvT, SLD, Emax, Jmax, st);
    else
      e = launch_gs_block_impl<T, 3, 1>(cl, wpc, g, t, cd, sc, ndir, dir_begin, dir_end, sweeps, f, phi, moments, TinvT, SLD, Emax, Jmax, st);
    if (e == cudaSuccess) {
      note_launch();
      if (status) *status = cl;
      return;
    }
    cudaGetLastError();
  }
  if (status) *status = 0;
}

template void launch_coarse_gs_block<double>(const Geom&, const LevelDev<double>&, const CellData&,
                                             const Schedule&, int, const int*, const int*, int,
                                             const double*, double*, double*, const double*,
                                             const double*, int, int, int, int, int, int, int, unsigned*, int*,
                                             int*, cudaStream_t);
template void launch_coarse_gs_block<float>(const Geom&, const LevelDev<float>&, const CellData&,
                                            const Schedule&, int, const int*, const int*, int,
                                            const float*, float*, float*, const float*,
                                            const float*, int, int, int, int, int, int, int, unsigned*, int*,
                                            int*, cudaStream_t);

template void launch_coarse_gs<double>(const Geom&, const LevelDev<double>&, const CellData&,
                                       const Schedule&, int, const int*, const int*, int,
                                       const double*, double*, double*, int*, cudaStream_t);
template void launch_coarse_gs<float>(const Geom&, const LevelDev<float>&, const CellData&,
                                      const Schedule&, int, const int*, const int*, int,
                                      const float*, float*, float*, int*, cudaStream_t);

}  // namespace amgt
