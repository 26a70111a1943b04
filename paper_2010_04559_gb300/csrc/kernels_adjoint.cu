// Gradients of a detector response R = g^T psi from the forward solution psi
// and the adjoint solution lambda of A^T lambda = g (A = L - S, Eq. complete
// and Sec. 4.2):
//
//   dR/dsigma_t[c] = -sum_q lambda_cq^T kron(N, M_q) psi_cq
//   dR/dsigma_s[c] =  lambda_c^T kron(N, S_f) psi_c
//                  =  sum_k f_deg(k) sum_{l,i} N_li PhiL[c,l,k] PhiP[c,i,k]
//   dR/df_n        =  sum_c sigma_s[c] sum_{k of degree n} sum_{l,i} N_li PhiL[c,l,k] PhiP[c,i,k]
//
// with the flux moments PhiP = psi X, PhiL = lambda X (S_f = X diag(f) X^T).
// FP64 throughout; one block per cell, block reductions, no atomics on the
// per-cell outputs.
#include "kernels.cuh"

namespace amgt {

namespace {

constexpr int kGradThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < (blockDim.x >> 5)) t = red[threadIdx.x];
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;  // valid in thread 0
}

// dsigt[c] for one cell per block; threads stride over the patches
template <int S, int A>
__global__ void __launch_bounds__(kGradThreads) grad_sigma_t_kernel(Geom g, const double* __restrict__ Mang,
                                                                    const double* __restrict__ psi,
                                                                    const double* __restrict__ lam,
                                                                    double* __restrict__ dsigt) {
  __shared__ double red[kGradThreads / 32];
  const long long c = blockIdx.x;
  const int nadof = g.nadof;
  double v = 0.0;
  for (int q = threadIdx.x; q < g.P; q += blockDim.x) {
    double mp[S][A];  // (M_q psi_cq)[i][m]
#pragma unroll
    for (int i = 0; i < S; ++i) {
      const double* pp = psi + (c * S + i) * nadof + q * A;
      double x[A];
#pragma unroll
      for (int d = 0; d < A; ++d) x[d] = pp[d];
#pragma unroll
      for (int m = 0; m < A; ++m) {
        double a = 0.0;
#pragma unroll
        for (int d = 0; d < A; ++d) a += Mang[((size_t)q * A + m) * A + d] * x[d];
        mp[i][m] = a;
      }
    }
#pragma unroll
    for (int l = 0; l < S; ++l) {
      const double* lp = lam + (c * S + l) * nadof + q * A;
#pragma unroll
      for (int m = 0; m < A; ++m) {
        double a = 0.0;
#pragma unroll
        for (int i = 0; i < S; ++i) a += g.Nmass[l * S + i] * mp[i][m];
        v += lp[m] * a;
      }
    }
  }
  const double t = block_sum(v, red);
  if (threadIdx.x == 0) dsigt[c] = -t;
}

// dsigs[c] per block and this block's contribution to dfn (added atomically)
template <int S>
__global__ void __launch_bounds__(kGradThreads) grad_moments_kernel(Geom g, int nmom, int N,
                                                                    const double* __restrict__ PhiP,
                                                                    const double* __restrict__ PhiL,
                                                                    const double* __restrict__ ftab,
                                                                    const int* __restrict__ fid,
                                                                    const double* __restrict__ sig_s,
                                                                    double* __restrict__ dsigs,
                                                                    double* __restrict__ dfn) {
  __shared__ double red[kGradThreads / 32];
  extern __shared__ double part[];  // [N+1] per-degree sums of this cell
  const long long c = blockIdx.x;
  const int sh = fid ? fid[c] : 0;
  const double* fmom = ftab + (size_t)sh * (N + 1);
  for (int n = threadIdx.x; n <= N; n += blockDim.x) part[n] = 0.0;
  __syncthreads();
  double vs = 0.0;
  for (int k = threadIdx.x; k < nmom; k += blockDim.x) {
    double t = 0.0;
#pragma unroll
    for (int l = 0; l < S; ++l) {
      double a = 0.0;
#pragma unroll
      for (int i = 0; i < S; ++i) a += g.Nmass[l * S + i] * PhiP[(c * S + i) * nmom + k];
      t += PhiL[(c * S + l) * nmom + k] * a;
    }
    int n = (int)sqrt((double)k);
    while (n * n > k) --n;
    while ((n + 1) * (n + 1) <= k) ++n;
    vs += fmom[n] * t;
    atomicAdd(&part[n], t);
  }
  const double ts = block_sum(vs, red);
  if (threadIdx.x == 0) dsigs[c] = ts;
  __syncthreads();
  const double ss = sig_s[c];
  for (int n = threadIdx.x; n <= N; n += blockDim.x)
    atomicAdd(&dfn[(size_t)sh * (N + 1) + n], ss * part[n]);
}

}  // namespace

void launch_grad_sigma_t(const Geom& g, const double* Mang, const double* psi, const double* lam,
                         double* dsigt, cudaStream_t st) {
  note_launch();
  const int grid = g.C;
  if (g.s == 4 && g.a == 3)
    grad_sigma_t_kernel<4, 3><<<grid, kGradThreads, 0, st>>>(g, Mang, psi, lam, dsigt);
  else if (g.s == 4)
    grad_sigma_t_kernel<4, 1><<<grid, kGradThreads, 0, st>>>(g, Mang, psi, lam, dsigt);
  else if (g.a == 3)
    grad_sigma_t_kernel<8, 3><<<grid, kGradThreads, 0, st>>>(g, Mang, psi, lam, dsigt);
  else
    grad_sigma_t_kernel<8, 1><<<grid, kGradThreads, 0, st>>>(g, Mang, psi, lam, dsigt);
}

void launch_grad_moments(const Geom& g, int nmom, int N, const double* PhiP, const double* PhiL,
                         const double* ftab, const int* fid, const double* sig_s, double* dsigs,
                         double* dfn, cudaStream_t st) {
  note_launch();
  const size_t smem = (size_t)(N + 1) * sizeof(double);
  if (g.s == 4)
    grad_moments_kernel<4><<<g.C, kGradThreads, smem, st>>>(g, nmom, N, PhiP, PhiL, ftab, fid,
                                                           sig_s, dsigs, dfn);
  else
    grad_moments_kernel<8><<<g.C, kGradThreads, smem, st>>>(g, nmom, N, PhiP, PhiL, ftab, fid,
                                                           sig_s, dsigs, dfn);
}

}  // namespace amgt
