// FP64-accurate scatter contraction from BF16 tensor-core products: the
// error-free splitting of Ozaki, Ogita, Oishi and Rump ("Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59, 2012), restated for tcgen05 BF16
// MMAs with FP32 accumulation.
//
// A row z of an FP64 matrix is scaled by mu = 2^e, the power of two just
// above max |z|, and cut into digit slices: t_0 = z / mu, then for each slice
// t <- t 2^b, d = rint(t), t <- t - d.  Every step is exact in FP64, every
// digit is an integer with |d_0| <= 2^b and |d_i| <= 2^(b-1) for i >= 1, so
// it is exact in BF16, and z = mu sum_i d_i 2^(-b(i+1)) + mu t 2^(-b nsl).
// For two sliced operands the product of slices i and j is a matrix of
// integer dot products bounded by K 2^(2b); while the accumulated bound
// stays at or below 2^24 the FP32 accumulator holds it exactly.  The host
// picks b and groups the slice pairs of each diagonal i + j = d under that
// bound; each group's exact integer sums are scaled by mu_r nu_c 2^(-b(d+2))
// (a power of two) and accumulated in FP64.
#include "kernels.cuh"

namespace amgt {

namespace {

constexpr int kSplitThreads = 256;

// z[l][k] of the block's row group: the per-cell mixed rows
// sig[c] sum_i Nm[l][i] x[c S + i][k] (MIX) or the rows themselves.
template <int S, bool MIX>
__device__ __forceinline__ void row_values(const double* __restrict__ x, long long r0, int K,
                                           int nrow, int k, double sig, const double* Nm,
                                           double (&z)[S]) {
  double v[S];
#pragma unroll
  for (int i = 0; i < S; ++i) v[i] = i < nrow ? x[(r0 + i) * (long long)K + k] : 0.0;
  if constexpr (MIX) {
#pragma unroll
    for (int l = 0; l < S; ++l) {
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < S; ++i) acc = __fma_rn(Nm[l * S + i], v[i], acc);
      z[l] = __dmul_rn(sig, acc);
    }
  } else {
#pragma unroll
    for (int l = 0; l < S; ++l) z[l] = v[l];
  }
}

// One block per group of S rows.  mu[r] receives the row scale 2^e,
// out[i * slice_stride + r K + k] the digit of slice i.
template <int S, bool MIX>
__global__ void __launch_bounds__(kSplitThreads) split_rows_kernel(
    long long rows, int K, const double* __restrict__ x, const double* __restrict__ sig,
    NmassArg nm, int nsl, int bits, double* __restrict__ mu, __nv_bfloat16* __restrict__ out,
    long long slice_stride) {
  __shared__ double red[kSplitThreads / 32][S];
  __shared__ double inv_s[S];
  __shared__ double Nm[S * S];
  const long long r0 = (long long)blockIdx.x * S;
  if (r0 >= rows) return;
  const int nrow = (int)min((long long)S, rows - r0);
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) Nm[e] = MIX ? nm.v[e] : 0.0;
  __syncthreads();
  const double sg = MIX ? sig[r0 / S] : 1.0;
  double m[S];
#pragma unroll
  for (int l = 0; l < S; ++l) m[l] = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double z[S];
    row_values<S, MIX>(x, r0, K, nrow, k, sg, Nm, z);
#pragma unroll
    for (int l = 0; l < S; ++l) m[l] = fmax(m[l], fabs(z[l]));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int l = 0; l < S; ++l) {
    double v = m[l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[warp][l] = v;
  }
  __syncthreads();
  if (threadIdx.x < S) {
    const int l = threadIdx.x;
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, red[w][l]);
    int e = 0;
    if (v > 0.0) frexp(v, &e);  // v = f 2^e, f in [0.5, 1): v < 2^e
    if (l < nrow) mu[r0 + l] = ldexp(1.0, e);
    inv_s[l] = ldexp(1.0, -e);
  }
  __syncthreads();
  double inv[S];
#pragma unroll
  for (int l = 0; l < S; ++l) inv[l] = inv_s[l];
  const double up = ldexp(1.0, bits);
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double z[S];
    row_values<S, MIX>(x, r0, K, nrow, k, sg, Nm, z);
#pragma unroll
    for (int l = 0; l < S; ++l) {
      if (l >= nrow) break;
      double t = z[l] * inv[l];
      __nv_bfloat16* o = out + (r0 + l) * (long long)K + k;
      for (int i = 0; i < nsl; ++i) {
        t *= up;
        const double d = rint(t);
        t -= d;
        o[i * slice_stride] = __double2bfloat16(d);
      }
    }
  }
}

// y[r][c] += sc mu[r] nu[c] P[r][c]  (sc mu nu is a power of two times sc)
__global__ void split_flush_kernel(long long M, int N, const float* __restrict__ P,
                                   const double* __restrict__ mu, const double* __restrict__ nu,
                                   double sc, double* __restrict__ y) {
  if ((N & 3) == 0) {
    const int n4 = N >> 2;
    const long long total = M * n4;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
      const long long r = idx / n4;
      const int c = (int)(idx - r * n4) * 4;
      const float4 p = __ldcs(reinterpret_cast<const float4*>(P + r * N + c));
      const double s = sc * mu[r];
      double2* yp = reinterpret_cast<double2*>(y + r * N + c);
      double2 a = yp[0], b = yp[1];
      a.x += (s * nu[c]) * (double)p.x;
      a.y += (s * nu[c + 1]) * (double)p.y;
      b.x += (s * nu[c + 2]) * (double)p.z;
      b.y += (s * nu[c + 3]) * (double)p.w;
      yp[0] = a;
      yp[1] = b;
    }
  } else {
    const long long total = M * N;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
      const long long r = idx / N;
      const int c = (int)(idx - r * N);
      y[idx] += (sc * mu[r] * nu[c]) * (double)P[idx];
    }
  }
}

}  // namespace

void launch_split_rows(long long rows, int K, int S, bool mix, const double* x,
                       const double* sig, const double* Nm, int nsl, int bits, double* mu,
                       __nv_bfloat16* out, long long slice_stride, cudaStream_t st) {
  note_launch();
  NmassArg nm{};
  if (mix)
    for (int e = 0; e < S * S; ++e) nm.v[e] = Nm[e];
  const long long groups = (rows + S - 1) / S;
  if (S == 8 && mix)
    split_rows_kernel<8, true><<<(unsigned)groups, kSplitThreads, 0, st>>>(
        rows, K, x, sig, nm, nsl, bits, mu, out, slice_stride);
  else if (S == 4 && mix)
    split_rows_kernel<4, true><<<(unsigned)groups, kSplitThreads, 0, st>>>(
        rows, K, x, sig, nm, nsl, bits, mu, out, slice_stride);
  else
    split_rows_kernel<4, false><<<(unsigned)((rows + 3) / 4), kSplitThreads, 0, st>>>(
        rows, K, x, sig, nm, nsl, bits, mu, out, slice_stride);
}

void launch_split_flush(long long M, int N, const float* P, const double* mu, const double* nu,
                        double sc, double* y, cudaStream_t st) {
  note_launch();
  const long long work = (N & 3) == 0 ? M * (N >> 2) : M * N;
  long long grid = (work + 255) / 256;
  if (grid > 152LL * 16) grid = 152LL * 16;
  if (grid < 1) grid = 1;
  split_flush_kernel<<<(unsigned)grid, 256, 0, st>>>(M, N, P, mu, nu, sc, y);
}

}  // namespace amgt
