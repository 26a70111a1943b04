// Transport kernels: the upwind DG sweep L^-1 (Sec. 3), the operator apply
// L x (Eq. complete), the source vector f, the angular transfers P / R = P^T
// (Sec. 4.1) and the scalar flux.
//
// Per (cell c, patch q) the unknowns form a block of s*a values with index
// l*a + m (spatial node l, angular function m).  The diagonal block of L is
//   K0_q + sigma_t(c) kron(N, M_q),
//   K0_q = sum_{outflow f} kron(Fown_f, A_{f,q}) - sum_xi kron(V_xi, A^xi_q),
// and an inflow face f couples to the upwind neighbour through
// kron(Fnb_f, A_{f,q}) with A_{f,q} = n_xi A^xi_q.  Fnb_f only links the face
// nodes of the two cells, with the Q1 face mass `facemass[xi]`.
#include "kernels.cuh"

namespace amgt {

namespace {

__device__ __forceinline__ int fnode(int j, int axis, int bit) {
  int lo = j & ((1 << axis) - 1);
  int hi = (j >> axis) << (axis + 1);
  return lo | (bit << axis) | hi;
}

// direction bits (1 = negative) of sweep direction d
template <int DIM>
__device__ __forceinline__ void dir_bits(int d, int neg[3]) {
  if (DIM == 2) {
    neg[0] = (d >> 1) & 1;
    neg[1] = d & 1;
    neg[2] = 0;
  } else {
    neg[0] = (d >> 2) & 1;
    neg[1] = (d >> 1) & 1;
    neg[2] = d & 1;
  }
}

// Adds sign * sum over inflow faces of kron(Fnb_f, A_{f,q}) psi_nb to acc.
template <class T, int DIM, int A>
__device__ __forceinline__ void upwind_term(const Geom& g, const T* __restrict__ Aax, int q,
                                            const T* __restrict__ psi, int c, const int jj[3],
                                            const int neg[3], T sign, T* acc) {
  constexpr int S = 1 << DIM;
  const int nadof = g.nadof;
  const int stride[3] = {1, g.nx, g.nx * g.ny};
#pragma unroll
  for (int xi = 0; xi < DIM; ++xi) {
    if (jj[xi] == 0) continue;  // domain boundary: inflow data lives in f
    const int own = neg[xi];    // side bit of this cell's inflow face
    const int cn = c + (own ? stride[xi] : -stride[xi]);
    const T* An = Aax + ((size_t)q * 3 + xi) * A * A;
    const T nsgn = own ? T(1) : T(-1);  // outward normal component
    const T* pn = psi + (long long)cn * S * nadof + q * A;
    T tv[S / 2][A];
#pragma unroll
    for (int j = 0; j < S / 2; ++j) {
      const int i = fnode(j, xi, 1 - own);
      T v[A];
#pragma unroll
      for (int d = 0; d < A; ++d) v[d] = pn[(long long)i * nadof + d];
#pragma unroll
      for (int m = 0; m < A; ++m) {
        T sacc = T(0);
#pragma unroll
        for (int d = 0; d < A; ++d) sacc += An[m * A + d] * v[d];
        tv[j][m] = nsgn * sacc;
      }
    }
#pragma unroll
    for (int jp = 0; jp < S / 2; ++jp) {
      const int l = fnode(jp, xi, own);
#pragma unroll
      for (int m = 0; m < A; ++m) {
        T sacc = T(0);
#pragma unroll
        for (int j = 0; j < S / 2; ++j) sacc += T(g.facemass[xi][jp][j]) * tv[j][m];
        acc[l * A + m] += sign * sacc;
      }
    }
  }
}

template <class T, int DIM, int A>
__global__ void __launch_bounds__(256) sweep_kernel(Geom g, LevelDev<T> t, CellData cd,
                                                    Schedule sc, const T* __restrict__ b,
                                                    T* __restrict__ psi) {
  constexpr int S = 1 << DIM;
  constexpr int SA = S * A;
  const int task = blockIdx.x;
  const int d = sc.task_dir[task], q0 = sc.task_q0[task], nq = sc.task_nq[task];
  int neg[3];
  dir_bits<DIM>(d, neg);
  const int nadof = g.nadof;
  for (int w = 0; w < sc.nlev; ++w) {
    const int beg = sc.level_off[w];
    const int work = (sc.level_off[w + 1] - beg) * nq;
    for (int idx = threadIdx.x; idx < work; idx += blockDim.x) {
      const int k = idx / nq;
      const int q = q0 + (idx - k * nq);
      const int packed = sc.cells[beg + k];
      const int jj[3] = {packed & 2047, (packed >> 11) & 2047, packed >> 22};
      const int ix = neg[0] ? g.nx - 1 - jj[0] : jj[0];
      const int iy = neg[1] ? g.ny - 1 - jj[1] : jj[1];
      const int iz = neg[2] ? g.nz - 1 - jj[2] : jj[2];
      const int c = ix + g.nx * (iy + g.ny * iz);
      T rhs[SA];
      const T* bp = b + (long long)c * S * nadof + q * A;
#pragma unroll
      for (int l = 0; l < S; ++l)
#pragma unroll
        for (int m = 0; m < A; ++m) rhs[l * A + m] = bp[(long long)l * nadof + m];
      upwind_term<T, DIM, A>(g, t.Aax, q, psi, c, jj, neg, T(-1), rhs);
      const T* Ki = t.Kinv + ((size_t)cd.mat[c] * g.P + q) * SA * SA;
      T* out = psi + (long long)c * S * nadof + q * A;
#pragma unroll
      for (int r = 0; r < SA; ++r) {
        T acc = T(0);
#pragma unroll
        for (int cc = 0; cc < SA; ++cc) acc += Ki[r * SA + cc] * rhs[cc];
        out[(long long)(r / A) * nadof + (r % A)] = acc;
      }
    }
    __syncthreads();
  }
}

template <class T, int DIM, int A>
__global__ void __launch_bounds__(256) apply_L_kernel(Geom g, LevelDev<T> t, CellData cd,
                                                      T alpha, T beta, const T* __restrict__ x,
                                                      T* __restrict__ y) {
  constexpr int S = 1 << DIM;
  constexpr int SA = S * A;
  const long long total = (long long)g.C * g.P;
  const int nadof = g.nadof;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / g.P);
    const int q = (int)(idx - (long long)c * g.P);
    int neg[3];
    dir_bits<DIM>(t.pdir[q], neg);
    const int ix = c % g.nx, iy = (c / g.nx) % g.ny, iz = c / (g.nx * g.ny);
    const int jj[3] = {neg[0] ? g.nx - 1 - ix : ix, neg[1] ? g.ny - 1 - iy : iy,
                       neg[2] ? g.nz - 1 - iz : iz};
    const T* xp = x + (long long)c * S * nadof + q * A;
    T xv[SA];
#pragma unroll
    for (int l = 0; l < S; ++l)
#pragma unroll
      for (int m = 0; m < A; ++m) xv[l * A + m] = xp[(long long)l * nadof + m];
    const T st = (T)cd.sigma_t[c];
    const T* K0 = t.K0 + (size_t)q * SA * SA;
    const T* Bq = t.B + (size_t)q * SA * SA;
    T acc[SA];
#pragma unroll
    for (int r = 0; r < SA; ++r) {
      T s1 = T(0), s2 = T(0);
#pragma unroll
      for (int cc = 0; cc < SA; ++cc) {
        s1 += K0[r * SA + cc] * xv[cc];
        s2 += Bq[r * SA + cc] * xv[cc];
      }
      acc[r] = s1 + st * s2;
    }
    upwind_term<T, DIM, A>(g, t.Aax, q, x, c, jj, neg, T(1), acc);
    T* out = y + (long long)c * S * nadof + q * A;
#pragma unroll
    for (int r = 0; r < SA; ++r) {
      T* o = out + (long long)(r / A) * nadof + (r % A);
      T v = alpha * acc[r];
      if (beta != T(0)) v += beta * (*o);
      *o = v;
    }
  }
}

// f[c*s+l][q*a+m] = q_c/(4 pi) mu_l w_qm + boundary inflow terms
template <class T>
__global__ void source_kernel(Geom g, const T* __restrict__ w, const T* __restrict__ Aw,
                              const int* __restrict__ octant, const double* __restrict__ qsrc,
                              const double* __restrict__ bval, const int* __restrict__ bkind,
                              const double* __restrict__ mu, const double* __restrict__ mf,
                              T* __restrict__ f) {
  const long long total = g.nsdof * g.nadof;
  const int a = g.a, s = g.s;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx / g.nadof;
    const int j = (int)(idx - r * g.nadof);
    const int c = (int)(r / s), l = (int)(r - (long long)c * s);
    const int q = j / a, m = j - q * a;
    double v = qsrc[c] / (4.0 * M_PI) * mu[l] * (double)w[j];
    const int ic[3] = {c % g.nx, (c / g.nx) % g.ny, c / (g.nx * g.ny)};
    const int n[3] = {g.nx, g.ny, g.nz};
    const int o = octant[q];
    const int negb[3] = {(o >> 2) & 1, (o >> 1) & 1, o & 1};
    for (int xi = 0; xi < g.dim; ++xi) {
      for (int side = 0; side < 2; ++side) {
        const int face = 2 * xi + side;
        if (bkind[face] != 1) continue;
        if (side == 0 ? ic[xi] != 0 : ic[xi] != n[xi] - 1) continue;
        // inflow iff the patch moves into the domain through this face
        const bool inflow = side == 0 ? (negb[xi] == 0) : (negb[xi] == 1);
        if (!inflow) continue;
        const double nsgn = side ? 1.0 : -1.0;
        v += -bval[face] * mf[face * s + l] * nsgn * (double)Aw[((size_t)q * 3 + xi) * a + m];
      }
    }
    f[idx] = (T)v;
  }
}

// phi[r] = sum_j psi[r][j] w[j]: one warp per row
template <class T>
__global__ void scalar_flux_kernel(long long nsdof, int nadof, const T* __restrict__ w,
                                   const T* __restrict__ psi, T* __restrict__ phi) {
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = warp; r < nsdof; r += nwarp) {
    double acc = 0.0;
    for (int j = lane; j < nadof; j += 32) acc += (double)psi[r * nadof + j] * (double)w[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) phi[r] = (T)acc;
  }
}

// rc[r][(c,d)] = sum_{f in children(c)} sum_k blk[f][k][d] rf[r][(f,k)]
template <class T>
__global__ void restrict_kernel(long long nsdof, int Pc, int a, int nadof_f, int nadof_c,
                                const int* __restrict__ cbeg, const int* __restrict__ cend,
                                const T* __restrict__ blk, const T* __restrict__ rf,
                                T* __restrict__ rc) {
  const long long total = nsdof * Pc;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx / Pc;
    const int c = (int)(idx - r * Pc);
    T acc[kMaxA] = {T(0), T(0), T(0)};
    for (int f = cbeg[c]; f < cend[c]; ++f) {
      for (int k = 0; k < a; ++k) {
        const T v = rf[r * nadof_f + f * a + k];
        for (int d = 0; d < a; ++d) acc[d] += blk[((size_t)f * a + k) * a + d] * v;
      }
    }
    for (int d = 0; d < a; ++d) rc[r * nadof_c + c * a + d] = acc[d];
  }
}

// xf[r][(f,k)] += sum_d blk[f][k][d] xc[r][(parent(f),d)]
template <class T>
__global__ void prolong_kernel(long long nsdof, int Pf, int a, int nadof_f, int nadof_c,
                               const int* __restrict__ parent, const T* __restrict__ blk,
                               const T* __restrict__ xc, T* __restrict__ xf) {
  const long long total = nsdof * Pf;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx / Pf;
    const int f = (int)(idx - r * Pf);
    const int p = parent[f];
    T v[kMaxA];
    for (int d = 0; d < a; ++d) v[d] = xc[r * nadof_c + p * a + d];
    for (int k = 0; k < a; ++k) {
      T acc = T(0);
      for (int d = 0; d < a; ++d) acc += blk[((size_t)f * a + k) * a + d] * v[d];
      xf[r * nadof_f + f * a + k] += acc;
    }
  }
}

int grid_for(long long total, int block) {
  long long g = (total + block - 1) / block;
  if (g > 152LL * 32) g = 152LL * 32;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

template <class T>
void launch_sweep(const Geom& g, const LevelDev<T>& t, const CellData& cd, const Schedule& sc,
                  const T* b, T* psi, cudaStream_t st) {
  note_launch();
  dim3 grid(sc.ntask), block(256);
  if (g.dim == 2 && g.a == 3) sweep_kernel<T, 2, 3><<<grid, block, 0, st>>>(g, t, cd, sc, b, psi);
  else if (g.dim == 2) sweep_kernel<T, 2, 1><<<grid, block, 0, st>>>(g, t, cd, sc, b, psi);
  else if (g.a == 3) sweep_kernel<T, 3, 3><<<grid, block, 0, st>>>(g, t, cd, sc, b, psi);
  else sweep_kernel<T, 3, 1><<<grid, block, 0, st>>>(g, t, cd, sc, b, psi);
}

template <class T>
void launch_apply_L(const Geom& g, const LevelDev<T>& t, const CellData& cd, T alpha, T beta,
                    const T* x, T* y, cudaStream_t st) {
  note_launch();
  const int grid = grid_for((long long)g.C * g.P, 256);
  if (g.dim == 2 && g.a == 3)
    apply_L_kernel<T, 2, 3><<<grid, 256, 0, st>>>(g, t, cd, alpha, beta, x, y);
  else if (g.dim == 2)
    apply_L_kernel<T, 2, 1><<<grid, 256, 0, st>>>(g, t, cd, alpha, beta, x, y);
  else if (g.a == 3)
    apply_L_kernel<T, 3, 3><<<grid, 256, 0, st>>>(g, t, cd, alpha, beta, x, y);
  else
    apply_L_kernel<T, 3, 1><<<grid, 256, 0, st>>>(g, t, cd, alpha, beta, x, y);
}

template <class T>
void launch_source(const Geom& g, const T* w, const T* Aw, const int* octant, const double* q,
                   const double* bval, const int* bkind, const double* mu, const double* mf,
                   T* f, cudaStream_t st) {
  note_launch();
  const int grid = grid_for(g.nsdof * g.nadof, 256);
  source_kernel<T><<<grid, 256, 0, st>>>(g, w, Aw, octant, q, bval, bkind, mu, mf, f);
}

template <class T>
void launch_scalar_flux(long long nsdof, int nadof, const T* w, const T* psi, T* phi,
                        cudaStream_t st) {
  note_launch();
  const int grid = grid_for(nsdof * 32, 256);
  scalar_flux_kernel<T><<<grid, 256, 0, st>>>(nsdof, nadof, w, psi, phi);
}

template <class T>
void launch_restrict(long long nsdof, int Pc, int a, int nadof_f, int nadof_c, const int* cbeg,
                     const int* cend, const T* blk, const T* rf, T* rc, cudaStream_t st) {
  note_launch();
  const int grid = grid_for(nsdof * Pc, 256);
  restrict_kernel<T><<<grid, 256, 0, st>>>(nsdof, Pc, a, nadof_f, nadof_c, cbeg, cend, blk, rf,
                                           rc);
}

template <class T>
void launch_prolong(long long nsdof, int Pf, int a, int nadof_f, int nadof_c, const int* parent,
                    const T* blk, const T* xc, T* xf, cudaStream_t st) {
  note_launch();
  const int grid = grid_for(nsdof * Pf, 256);
  prolong_kernel<T><<<grid, 256, 0, st>>>(nsdof, Pf, a, nadof_f, nadof_c, parent, blk, xc, xf);
}

#define AMGT_INST(T)                                                                          \
  template void launch_sweep<T>(const Geom&, const LevelDev<T>&, const CellData&,             \
                                const Schedule&, const T*, T*, cudaStream_t);                 \
  template void launch_apply_L<T>(const Geom&, const LevelDev<T>&, const CellData&, T, T,     \
                                  const T*, T*, cudaStream_t);                                \
  template void launch_source<T>(const Geom&, const T*, const T*, const int*, const double*,  \
                                 const double*, const int*, const double*, const double*, T*, \
                                 cudaStream_t);                                               \
  template void launch_scalar_flux<T>(long long, int, const T*, const T*, T*, cudaStream_t);  \
  template void launch_restrict<T>(long long, int, int, int, int, const int*, const int*,     \
                                   const T*, const T*, T*, cudaStream_t);                     \
  template void launch_prolong<T>(long long, int, int, int, int, const int*, const T*,        \
                                  const T*, T*, cudaStream_t);
AMGT_INST(double)
AMGT_INST(float)
#undef AMGT_INST

}  // namespace amgt
