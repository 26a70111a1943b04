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

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace amgt {

namespace {

__device__ __forceinline__ int fnode(int j, int axis, int bit) {
  int lo = j & ((1 << axis) - 1);
  int hi = (j >> axis) << (axis + 1);
  return lo | (bit << axis) | hi;
}
__device__ __forceinline__ int fcompress(int l, int axis) {
  int lo = l & ((1 << axis) - 1);
  int hi = (l >> (axis + 1)) << axis;
  return lo | hi;
}

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
              const T* xf = t.XFt;  // [nm][nadof]
              for (int kk = 0; kk < nm; ++kk) G += xf[(long long)kk * nadof + q * A + m] * __ldcg(Phi + l * nm + kk);
            }
            const T* Sq = t.Sqq + (size_t)q * A * A;
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

template void launch_coarse_gs<double>(const Geom&, const LevelDev<double>&, const CellData&,
                                       const Schedule&, int, const int*, const int*, int,
                                       const double*, double*, double*, int*, cudaStream_t);
template void launch_coarse_gs<float>(const Geom&, const LevelDev<float>&, const CellData&,
                                      const Schedule&, int, const int*, const int*, int,
                                      const float*, float*, float*, int*, cudaStream_t);

}  // namespace amgt
