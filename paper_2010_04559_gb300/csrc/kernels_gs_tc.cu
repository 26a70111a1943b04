// Coarse-mesh block Gauss-Seidel (Sec. 4.2), direction-blocked form, with the
// dense contractions on tensor cores.  Same iteration as coarse_gs_block_kernel
// (see kernels_gs.cu): per cell c and sweep direction d,
//   rhs_c = f_c - upwind_c + sigma_s N (x) (X_d F Phi_c - S_dd^{L+D} x_c^old)
//   x_c^new = Tinv[mat(c), d] rhs_c,     Phi_c += X_d^T (x_c^new - x_c^old).
// A thread block handles NC = 8 cells of a wavefront level at once and stacks
// them so that each table is a shared-memory matrix operand read once per
// level:
//   BUF[8s x J]  = PHI[8s x nm] XF^T[nm x J] - XOLD[8s x J] SL^T[J x J]
//   XNEW[E x 8]  = Tinv_mat[E x E] RHS[E x 8]     (one pass per material present)
//   DPHI[8s x nm] = DELTA[8s x J] X_d[J x nm]
// with mma.sync m16n8k8 on TF32 operands split in high and low parts
// (a = a_hi + a_lo; a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi), which keeps
// close to FP32 accuracy.  Wavefront levels are separated by the cluster
// barrier; blocks of a 16-block cluster take consecutive groups of 8 cells.
#include <cooperative_groups.h>

#include <algorithm>

#include "gs_common.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace amgt {

namespace {

constexpr int NC = 8;      // cells per block per level (the MMA N dimension)
constexpr int WARPS = 8;


__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// d += A B with A read as A(row, col) = pa[row * lda + col] (16 x 8 tile at
// (m0, k0)) and B as B(k, n) = pb[n * ldb + k] (8 x 8 tile at (k0, n0)),
// three-pass split TF32.
// three independent accumulators (d[0]: lo*hi, d[1]: hi*lo, d[2]: hi*hi) keep
// the tensor-core pipeline busy; the caller sums them
__device__ __forceinline__ void mma_split3(float (&d)[3][4], const float* pa, int lda, int m0,
                                           int k0, const float* pb, int ldb, int n0, int lane) {
  const int g = lane >> 2, t = lane & 3;
  float af[4] = {pa[(m0 + g) * lda + k0 + t], pa[(m0 + g + 8) * lda + k0 + t],
                 pa[(m0 + g) * lda + k0 + t + 4], pa[(m0 + g + 8) * lda + k0 + t + 4]};
  float bf[2] = {pb[(n0 + g) * ldb + k0 + t], pb[(n0 + g) * ldb + k0 + t + 4]};
  uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) split_tf32(af[i], ah[i], al[i]);
#pragma unroll
  for (int i = 0; i < 2; ++i) split_tf32(bf[i], bh[i], bl[i]);
  mma_tf32(d[0], al, bh);
  mma_tf32(d[1], ah, bl);
  mma_tf32(d[2], ah, bh);
}
__device__ __forceinline__ void mma_split(float (&d)[4], const float* pa, int lda, int m0, int k0,
                                          const float* pb, int ldb, int n0, int lane) {
  const int g = lane >> 2, t = lane & 3;
  float af[4] = {pa[(m0 + g) * lda + k0 + t], pa[(m0 + g + 8) * lda + k0 + t],
                 pa[(m0 + g) * lda + k0 + t + 4], pa[(m0 + g + 8) * lda + k0 + t + 4]};
  float bf[2] = {pb[(n0 + g) * ldb + k0 + t], pb[(n0 + g) * ldb + k0 + t + 4]};
  uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) split_tf32(af[i], ah[i], al[i]);
#pragma unroll
  for (int i = 0; i < 2; ++i) split_tf32(bf[i], bh[i], bl[i]);
  mma_tf32(d, al, bh);
  mma_tf32(d, ah, bl);
  mma_tf32(d, ah, bh);
}

struct TcLayout {
  int E, J, nmK;      // entries, angular DOF of the direction, moments padded to 8
  int Ep, Kp, Jp;     // padded row strides
};

template <int DIM, int A>
__global__ void __launch_bounds__(WARPS * 32) coarse_gs_tc_kernel(
    Geom g, LevelDev<float> t, CellData cd, Schedule sc, int ndir, const int* __restrict__ dir_begin,
    const int* __restrict__ dir_end, int sweeps, const float* __restrict__ f,
    float* __restrict__ psi, float* __restrict__ mom, const float* __restrict__ TinvT,
    const float* __restrict__ SLD, int Emax, int Jmax, int nmat, int Ep, int Kp, int Jp, int nmK) {
  constexpr int S = 1 << DIM;
  constexpr int HS = S / 2;
  constexpr int R = NC * S;  // stacked rows (cell, spatial node)
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) float sm[];
  const int nm = t.nmom;
  const int nadof = g.nadof;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rank = (int)cluster.block_rank();
  const int nblk = (int)cluster.num_blocks();
  // shared layout
  float* Tin = sm;                                   // [nmat][Emax][Ep]   A of the solve
  float* XFr = Tin + (size_t)nmat * Emax * Ep;       // [Jmax][Kp]         B of the source
  float* SLr = XFr + (size_t)Jmax * Kp;              // [Jmax][Jp]         B of the self-scatter
  float* Xk = SLr + (size_t)Jmax * Jp;               // [nmK][Jp]          B of the moment update
  float* PHI = Xk + (size_t)nmK * Jp;                // [R][Kp]            moments of the cells
  float* XO = PHI + (size_t)R * Kp;                  // [R][Jp]            old values, then delta
  float* BUF = XO + (size_t)R * Jp;                  // [R][Jp]            source before the mixing
  float* RHS = BUF + (size_t)R * Jp;                 // [NC][Ep]           right-hand sides
  float* XN = RHS + (size_t)NC * Ep;                 // [NC][Ep]           new values
  float* UPW = XN + (size_t)NC * Ep;                 // [NC][DIM][HS][Jmax] neighbour faces
  int* cinfo = reinterpret_cast<int*>(UPW + (size_t)NC * DIM * HS * Jmax);  // [NC] cell or -1
  int* cmat = cinfo + NC;                                                   // [NC]
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
      // ---- stage the direction's tables (previous level ended with a cluster barrier)
      for (int mt = 0; mt < nmat; ++mt) {
        const float* src = TinvT + ((size_t)mt * ndir + d) * Emax * Emax;  // [col][row]
        float* dst = Tin + (size_t)mt * Emax * Ep;
        for (int i = threadIdx.x; i < Emax * Emax; i += blockDim.x) {
          const int col = i / Emax, row = i - col * Emax;
          dst[(size_t)row * Ep + col] = (row < E && col < E) ? src[i] : 0.f;
        }
      }
      for (int i = threadIdx.x; i < Jmax * Kp; i += blockDim.x) {
        const int j = i / Kp, k = i - j * Kp;
        XFr[i] = (j < J && k < nm) ? t.XFt[(long long)k * nadof + qb * A + j] : 0.f;
      }
      for (int i = threadIdx.x; i < Jmax * Jp; i += blockDim.x) {
        const int j = i / Jp, j2 = i - j * Jp;
        SLr[i] = (j < J && j2 < J) ? SLD[((size_t)d * Jmax + j) * Jmax + j2] : 0.f;
      }
      for (int i = threadIdx.x; i < nmK * Jp; i += blockDim.x) {
        const int k = i / Jp, j = i - k * Jp;
        Xk[i] = (k < nm && j < J) ? t.X[(long long)(qb * A + j) * nm + k] : 0.f;
      }
      __syncthreads();
      for (int w = 0; w < sc.nlev; ++w) {
        int cnt;
        if (DIM == 2) cnt = min(w, g.ny - 1) - max(0, w - (g.nx - 1)) + 1;
        else cnt = sc.level_off[w + 1] - sc.level_off[w];
        for (int base = rank * NC; base < cnt; base += nblk * NC) {
          // ---- cells of this block and their data
          if (threadIdx.x < NC) {
            const int k = base + threadIdx.x;
            int c = -1, mt = 0;
            if (k < cnt) {
              int j0, j1, j2c;
              if (DIM == 2) {
                j1 = max(0, w - (g.nx - 1)) + k;
                j0 = w - j1;
                j2c = 0;
              } else {
                const int packed = sc.cells[sc.level_off[w] + k];
                j0 = packed & 2047; j1 = (packed >> 11) & 2047; j2c = packed >> 22;
              }
              const int ix = n0 ? g.nx - 1 - j0 : j0;
              const int iy = n1 ? g.ny - 1 - j1 : j1;
              const int iz = n2 ? g.nz - 1 - j2c : j2c;
              c = ix + g.nx * (iy + g.ny * iz);
              mt = cd.mat[c];
            }
            cinfo[threadIdx.x] = c;
            cmat[threadIdx.x] = mt;
          }
          __syncthreads();
          // neighbour face values of every cell
          for (int i = threadIdx.x; i < NC * DIM * HS * J; i += blockDim.x) {
            const int cl = i / (DIM * HS * J);
            const int rem = i - cl * DIM * HS * J;
            const int xi = rem / (HS * J);
            const int rem2 = rem - xi * HS * J;
            const int jn = rem2 / J, j = rem2 - jn * J;
            const int c = cinfo[cl];
            float v = 0.f;
            if (c >= 0) {
              const int own = xi == 0 ? n0 : (xi == 1 ? n1 : n2);
              const int ic = xi == 0 ? c % g.nx : (xi == 1 ? (c / g.nx) % g.ny : c / (g.nx * g.ny));
              const int ncx = xi == 0 ? g.nx : (xi == 1 ? g.ny : g.nz);
              const bool has = own ? (ic < ncx - 1) : (ic > 0);
              if (has) {
                const int strd = xi == 0 ? 1 : (xi == 1 ? g.nx : g.nx * g.ny);
                const int cn = c + (own ? strd : -strd);
                const int node = gsx::fnode(jn, xi, 1 - own);
                v = __ldcg(psi + ((long long)cn * S + node) * nadof + qb * A + j);
              }
            }
            UPW[((cl * DIM + xi) * HS + jn) * Jmax + j] = v;
          }
          // old values and moments
          for (int i = threadIdx.x; i < R * J; i += blockDim.x) {
            const int row = i / J, j = i - row * J;
            const int cl = row / S, l = row - cl * S;
            const int c = cinfo[cl];
            XO[row * Jp + j] = c >= 0 ? __ldcg(psi + ((long long)c * S + l) * nadof + qb * A + j) : 0.f;
          }
          for (int i = threadIdx.x; i < R * Kp; i += blockDim.x) {
            const int row = i / Kp, k = i - row * Kp;
            const int cl = row / S;
            const int c = cinfo[cl];
            PHI[i] = (c >= 0 && k < nm) ? __ldcg(mom + (long long)c * S * nm + (row - cl * S) * nm + k) : 0.f;
          }
          __syncthreads();
          // ---- rhs = f - upwind (one entry per thread)
          for (int i = threadIdx.x; i < NC * E; i += blockDim.x) {
            const int cl = i / E, e = i - cl * E;
            const int c = cinfo[cl];
            float val = 0.f;
            if (c >= 0) {
              const int l = e / J, j = e - l * J;
              const int q = qb + j / A, m = j % A;
              val = f[((long long)c * S + l) * nadof + qb * A + j];
#pragma unroll
              for (int xi = 0; xi < DIM; ++xi) {
                const int own = xi == 0 ? n0 : (xi == 1 ? n1 : n2);
                if (((l >> xi) & 1) != own) continue;
                const float* An = t.Aax + ((size_t)q * 3 + xi) * A * A + m * A;
                const int jp = gsx::fcompress(l, xi);
                const int jb = (j / A) * A;
                float acc = 0.f;
#pragma unroll
                for (int jn = 0; jn < HS; ++jn) {
                  const float* nv = UPW + ((cl * DIM + xi) * HS + jn) * Jmax + jb;
                  float sacc = 0.f;
#pragma unroll
                  for (int dd = 0; dd < A; ++dd) sacc += An[dd] * nv[dd];
                  acc += (float)g.facemass[xi][jp][jn] * sacc;
                }
                val -= (own ? 1.f : -1.f) * acc;
              }
            }
            RHS[cl * Ep + e] = val;
          }
          // ---- BUF = PHI XF^T - XO SL^T on tensor cores: R x J tiles of 16 x 8
          {
            const int mt_n = R / 16, nt_n = J / 8;
            for (int tile = warp; tile < mt_n * nt_n; tile += WARPS) {
              const int m0 = (tile / nt_n) * 16, n0t = (tile % nt_n) * 8;
              float da[3][4] = {}, dn[3][4] = {};
              for (int k0 = 0; k0 < nmK; k0 += 8) mma_split3(da, PHI, Kp, m0, k0, XFr, Kp, n0t, lane);
              for (int k0 = 0; k0 < J; k0 += 8) mma_split3(dn, XO, Jp, m0, k0, SLr, Jp, n0t, lane);
              const int gq = lane >> 2, tq = lane & 3;
              float o[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) o[i] = (da[0][i] + da[1][i] + da[2][i]) - (dn[0][i] + dn[1][i] + dn[2][i]);
              BUF[(m0 + gq) * Jp + n0t + 2 * tq] = o[0];
              BUF[(m0 + gq) * Jp + n0t + 2 * tq + 1] = o[1];
              BUF[(m0 + gq + 8) * Jp + n0t + 2 * tq] = o[2];
              BUF[(m0 + gq + 8) * Jp + n0t + 2 * tq + 1] = o[3];
            }
          }
          __syncthreads();
          // ---- RHS += sigma_s N (x) BUF
          for (int i = threadIdx.x; i < NC * E; i += blockDim.x) {
            const int cl = i / E, e = i - cl * E;
            const int c = cinfo[cl];
            if (c < 0) continue;
            const int l = e / J, j = e - l * J;
            float acc = 0.f;
#pragma unroll
            for (int ii = 0; ii < S; ++ii) acc += (float)g.Nmass[l * S + ii] * BUF[(cl * S + ii) * Jp + j];
            RHS[cl * Ep + e] += (float)cd.sigma_s[c] * acc;
          }
          __syncthreads();
          // ---- XNEW = Tinv_mat RHS: E x 8 in 16 x 8 tiles, one pass per material present
          {
            const int mt_n = E / 16;
            for (int tile = warp; tile < mt_n; tile += WARPS) {
              const int m0 = tile * 16;
              float dd[2][3][4] = {};
              const int gq = lane >> 2, tq = lane & 3;
              for (int mt = 0; mt < nmat; ++mt) {
                bool present = false;
#pragma unroll
                for (int cl = 0; cl < NC; ++cl) present |= (cinfo[cl] >= 0 && cmat[cl] == mt);
                if (!present) continue;
                // B column of cell gq: masked unless it has material mt
                const bool mine = cinfo[gq] >= 0 && cmat[gq] == mt;
                const float* Tm = Tin + (size_t)mt * Emax * Ep;
                for (int k0 = 0; k0 < E; k0 += 8) {
                  float af[4] = {Tm[(m0 + gq) * Ep + k0 + tq], Tm[(m0 + gq + 8) * Ep + k0 + tq],
                                 Tm[(m0 + gq) * Ep + k0 + tq + 4], Tm[(m0 + gq + 8) * Ep + k0 + tq + 4]};
                  float bf[2] = {mine ? RHS[gq * Ep + k0 + tq] : 0.f,
                                 mine ? RHS[gq * Ep + k0 + tq + 4] : 0.f};
                  uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
                  for (int i2 = 0; i2 < 4; ++i2) split_tf32(af[i2], ah[i2], al[i2]);
#pragma unroll
                  for (int i2 = 0; i2 < 2; ++i2) split_tf32(bf[i2], bh[i2], bl[i2]);
                  const int h = (k0 >> 3) & 1;  // alternate two K halves
                  mma_tf32(dd[h][0], al, bh);
                  mma_tf32(dd[h][1], ah, bl);
                  mma_tf32(dd[h][2], ah, bh);
                }
              }
              float dacc[4];
#pragma unroll
              for (int i = 0; i < 4; ++i)
                dacc[i] = (dd[0][0][i] + dd[1][0][i]) + (dd[0][1][i] + dd[1][1][i]) + (dd[0][2][i] + dd[1][2][i]);
              // C(entry, cell): rows m0 + gq (+8), columns 2 tq (+1)
              XN[(2 * tq) * Ep + m0 + gq] = dacc[0];
              XN[(2 * tq + 1) * Ep + m0 + gq] = dacc[1];
              XN[(2 * tq) * Ep + m0 + gq + 8] = dacc[2];
              XN[(2 * tq + 1) * Ep + m0 + gq + 8] = dacc[3];
            }
          }
          __syncthreads();
          // ---- store psi, delta = xnew - xold into XO
          for (int i = threadIdx.x; i < R * J; i += blockDim.x) {
            const int row = i / J, j = i - row * J;
            const int cl = row / S, l = row - cl * S;
            const int c = cinfo[cl];
            const float xn = XN[cl * Ep + l * J + j];
            if (c >= 0) psi[((long long)c * S + l) * nadof + qb * A + j] = xn;
            XO[row * Jp + j] = c >= 0 ? xn - XO[row * Jp + j] : 0.f;
          }
          __syncthreads();
          // ---- PHI += DELTA X_d: R x nmK tiles
          {
            const int mt_n = R / 16, nt_n = nmK / 8;
            for (int tile = warp; tile < mt_n * nt_n; tile += WARPS) {
              const int m0 = (tile / nt_n) * 16, n0t = (tile % nt_n) * 8;
              float d3[3][4] = {};
              for (int k0 = 0; k0 < J; k0 += 8) mma_split3(d3, XO, Jp, m0, k0, Xk, Jp, n0t, lane);
              float dacc[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) dacc[i] = d3[0][i] + d3[1][i] + d3[2][i];
              const int gq = lane >> 2, tq = lane & 3;
              const int rows[2] = {m0 + gq, m0 + gq + 8};
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int row = rows[h];
                const int cl = row / S, l = row - cl * S;
                const int c = cinfo[cl];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                  const int k = n0t + 2 * tq + u;
                  if (c >= 0 && k < nm)
                    mom[(long long)c * S * nm + l * nm + k] = PHI[row * Kp + k] + dacc[2 * h + u];
                }
              }
            }
          }
          __syncthreads();
        }
        cluster.sync();
      }
    }
  }
}

}  // namespace

// sizes of the shared-memory layout above (floats)
static size_t gs_tc_smem_floats(int nmat, int Emax, int Jmax, int s, int dim, int Ep, int Kp,
                                int Jp, int nmK) {
  const int R = NC * s;
  return (size_t)nmat * Emax * Ep + (size_t)Jmax * Kp + (size_t)Jmax * Jp + (size_t)nmK * Jp +
         (size_t)R * Kp + 2 * (size_t)R * Jp + 2 * (size_t)NC * Ep +
         (size_t)NC * dim * (s / 2) * Jmax + 2 * NC;
}

int launch_coarse_gs_tc(const Geom& g, const LevelDev<float>& t, const CellData& cd,
                        const Schedule& sc, int ndir, const int* dir_begin, const int* dir_end,
                        const int* hdir_begin, const int* hdir_end, int sweeps, const float* f,
                        float* phi, float* moments, const float* TinvT, const float* SLD, int Emax,
                        int Jmax, int nmat, int cluster_req, cudaStream_t st) {
  // shape limits of the tensor-core form: every direction's J a multiple of 8,
  // E = s J a multiple of 16, stacked rows 8 s a multiple of 16
  for (int d = 0; d < ndir; ++d) {
    const int J = (hdir_end[d] - hdir_begin[d]) * g.a;
    if (J % 8 != 0 || (g.s * J) % 16 != 0) return -1;
  }
  if ((NC * g.s) % 16 != 0 || t.nmom > 128) return -1;
  const int nmK = ((t.nmom + 7) / 8) * 8;
  // padded strides: rows of 16x8 A tiles and 8x8 B tiles hit distinct banks when
  // the stride is 4 (mod 32) words
  auto pad4 = [](int n) { int p = ((n + 3) / 4) * 4; while (p % 32 != 4) p += 4; return p; };
  const int Ep = pad4(Emax), Kp = pad4(nmK), Jp = pad4(Jmax);
  const size_t smem = gs_tc_smem_floats(nmat, Emax, Jmax, g.s, g.dim, Ep, Kp, Jp, nmK) * sizeof(float);
  if (smem > 220 * 1024) return -2;
  int sizes[3] = {16, 8, 1};
  if (cluster_req > 0) sizes[0] = sizes[1] = sizes[2] = cluster_req;
  for (int cl : sizes) {
    auto kern = (g.dim == 2) ? (g.a == 3 ? coarse_gs_tc_kernel<2, 3> : coarse_gs_tc_kernel<2, 1>)
                             : (g.a == 3 ? coarse_gs_tc_kernel<3, 3> : coarse_gs_tc_kernel<3, 1>);
    if (allow_max_smem(kern) !=
        cudaSuccess) {
      cudaGetLastError();
      return -3;
    }
    if (cl > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(WARPS * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl < 1) {
      cudaGetLastError();
      continue;
    }
    if (cudaLaunchKernelEx(&cfg, kern, g, t, cd, sc, ndir, dir_begin, dir_end, sweeps, f, phi,
                           moments, TinvT, SLD, Emax, Jmax, nmat, Ep, Kp, Jp, nmK) == cudaSuccess) {
      note_launch();
      return cl;
    }
    cudaGetLastError();
  }
  return -4;
}

}  // namespace amgt
