// FP64-accurate scatter contraction from BF16 tensor-core products: the
// error-free splitting of Ozaki, Ogita, Oishi and Rump ("Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59, 2012), restated for tcgen05 BF16
// MMAs with FP32 accumulation.
//
// A row z of an FP64 matrix is scaled by mu = 2^e, a power of two above
// max |z|, and cut into nsl digit slices of b bits: z / mu rounded to a
// multiple of 2^(-b nsl) is sum_i d_i 2^(-b(i+1)) with integer digits,
// |d_0| <= 2^b and |d_i| <= 2^(b-1) for i >= 1 (balanced), exact in BF16.
// For two sliced operands the product of slices i and j is a matrix of
// integer dot products bounded by K 2^(2b); while the accumulated bound
// stays at or below 2^24 the FP32 accumulator holds it exactly.  The host
// picks b and groups the slice pairs of each leading diagonal i + j = d under
// that bound; each group's exact integer sums are scaled by mu_r nu_c
// 2^(-b(d+2)) (a power of two) and accumulated in FP64.  The trailing
// diagonals, whose sum lies 2^(-b d_t) below the leading term, are summed on
// the tensor cores in FP32 by Horner's rule (each diagonal's first product
// adds 2^(-b) times the sum of the less significant ones) and accumulated in
// FP64 once.
#include <climits>

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

// rint(z 2^s) (round half to even) from the FP64 bit pattern of z by integer
// operations, for |z 2^s| < 2^62; subnormal z by the FP64 route
__device__ __forceinline__ long long scaled_rint(double z, int s) {
  const long long b = __double_as_longlong(z);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return (b << 1) == 0 ? 0 : __double2ll_rn(ldexp(z, s));
  const long long m = (b & 0xfffffffffffffll) | (1ll << 52);
  const int sh = 1075 - ex - s;  // z 2^s = m 2^(-sh)
  long long t;
  if (sh <= 0) {
    t = m << (-sh);
  } else if (sh >= 54) {
    t = 0;  // |z 2^s| < 1/2
  } else {
    const long long q = m >> sh, rem = m & ((1ll << sh) - 1), half = 1ll << (sh - 1);
    t = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
  }
  return b < 0 ? -t : t;
}

// One block per group of S rows.  mu[r] receives the row scale 2^e,
// out[i * slice_stride + r K + k] the digit of slice i.
//
// The scale comes from a bound rather than the exact maximum: with m_i the
// largest |x| of input row i (an integer maximum of the bit patterns, no FP64
// arithmetic), |z_l| <= |sig| sum_i |N_li| m_i, and 2^e is the power of two
// above that bound (at most a bit is lost where rows cancel).  The digits are
// then taken in integer arithmetic: T = rint(z 2^(bits nsl - e)) is an exact
// integer with |T| <= 2^(bits nsl); from the least significant end, the
// balanced remainder r in [-2^(bits-1), 2^(bits-1)) of T modulo 2^bits is a
// digit and (T - r) / 2^bits (an exact shift) carries on; what is left after
// nsl - 1 digits is the leading digit, |d_0| <= 2^bits.  GB300's FP64 rate
// makes the FP64 form of this (three FP64 operations per digit) the slowest
// step of the split scatter; here each unknown costs only the mixing in FP64:
// the power-of-two scaling and the rounding to T work on the FP64 bit
// pattern in integer arithmetic, and the digits convert to BF16 through
// 32-bit integers.  A row whose bound is not finite gets mu = NaN, so the
// product carries it.
template <int S, bool MIX>
__global__ void __launch_bounds__(kSplitThreads) split_rows_kernel(
    long long rows, int K, const double* __restrict__ x, const double* __restrict__ sig,
    NmassArg nm, int nsl, int bits, double* __restrict__ mu, __nv_bfloat16* __restrict__ out,
    long long slice_stride) {
  __shared__ unsigned long long red[kSplitThreads / 32][S];
  __shared__ int sh_s[S];  // bits nsl - e, or INT_MIN for a row that is not finite
  __shared__ double Nm[S * S];
  const long long r0 = (long long)blockIdx.x * S;
  if (r0 >= rows) return;
  const int nrow = (int)min((long long)S, rows - r0);
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) Nm[e] = MIX ? nm.v[e] : 0.0;
  const double sg = MIX ? sig[r0 / S] : 1.0;
  // largest |x| of each input row as bit patterns (monotone for |x|)
  unsigned long long m[S];
#pragma unroll
  for (int i = 0; i < S; ++i) m[i] = 0ull;
  const unsigned long long* xb = reinterpret_cast<const unsigned long long*>(x);
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
#pragma unroll
    for (int i = 0; i < S; ++i)
      if (i < nrow) {
        const unsigned long long v = xb[(r0 + i) * (long long)K + k] & 0x7fffffffffffffffull;
        m[i] = v > m[i] ? v : m[i];
      }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    unsigned long long v = m[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < S) {
    const int l = threadIdx.x;
    double bound = 0.0;
    for (int i = 0; i < S; ++i) {
      unsigned long long v = 0ull;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = red[w][i] > v ? red[w][i] : v;
      const double mi = __longlong_as_double((long long)v);
      if (MIX) bound += fabs(Nm[l * S + i]) * mi;
      else if (i == l) bound = mi;
    }
    bound *= fabs(sg);
    int e = 0;
    if (bound > 0.0) frexp(bound, &e);  // bound = f 2^e, f in [0.5, 1)
    if (l < nrow) mu[r0 + l] = isfinite(bound) ? ldexp(1.0, e) : __longlong_as_double(0x7ff8000000000000ll);
    sh_s[l] = isfinite(bound) ? bits * nsl - e : INT_MIN;
  }
  __syncthreads();
  int shl[S];
#pragma unroll
  for (int l = 0; l < S; ++l) shl[l] = sh_s[l];
  const long long half = 1ll << (bits - 1), mask = (1ll << bits) - 1;
  // two adjacent columns per thread, stored as BF16 pairs (K and the slice
  // stride are even)
  const long long ss2 = slice_stride / 2;
  for (int k = 2 * threadIdx.x; k < K; k += 2 * blockDim.x) {
    double z0[S], z1[S];
    row_values<S, MIX>(x, r0, K, nrow, k, sg, Nm, z0);
    row_values<S, MIX>(x, r0, K, nrow, k + 1, sg, Nm, z1);
#pragma unroll
    for (int l = 0; l < S; ++l) {
      if (l >= nrow) break;
      // T = rint(z 2^(bits nsl - e)), exact (the scale is a power of two)
      long long T0 = shl[l] == INT_MIN ? 0 : scaled_rint(z0[l], shl[l]);
      long long T1 = shl[l] == INT_MIN ? 0 : scaled_rint(z1[l], shl[l]);
      __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(out + (r0 + l) * (long long)K + k);
      for (int i = nsl - 1; i > 0; --i) {
        const long long d0 = ((T0 + half) & mask) - half;
        const long long d1 = ((T1 + half) & mask) - half;
        T0 = (T0 - d0) >> bits;
        T1 = (T1 - d1) >> bits;
        // digits of at most 8 bits: 32-bit integer to float conversions
        o[i * ss2] = __floats2bfloat162_rn((float)(int)d0, (float)(int)d1);
      }
      o[0] = __floats2bfloat162_rn((float)(int)T0, (float)(int)T1);
    }
  }
}

// p 2^k as FP64, exactly, by integer operations on the FP32 bit pattern
// (zero and normal results; the rest by the FP64 route)
__device__ __forceinline__ double scaled_f2d(float p, int k) {
  const unsigned u = __float_as_uint(p);
  if ((u & 0x7fffffffu) == 0u) return 0.0;
  const int ex = (int)((u >> 23) & 0xffu);
  const int e = ex - 127 + 1023 + k;
  if (ex == 0 || ex == 255 || e <= 0 || e >= 2047) return ldexp((double)p, k);
  return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                          ((unsigned long long)e << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}
// the exponent of a finite power of two, or INT_MIN for anything else
__device__ __forceinline__ int pow2_exp(double v) {
  const long long b = __double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7ff);
  return ((b & 0xfffffffffffffll) == 0 && ex != 0 && ex != 0x7ff) ? ex - 1023 : INT_MIN;
}

// y[r][c] += sc mu[r] nu[c] P[r][c]  (sc mu nu is a power of two times sc,
// so each product is exact and only the sum rounds).  A block per row at a
// time: no index division, one row scale per row.  Where sc mu[r] and nu[c]
// are powers of two (the split form's scales; sc = +-2^-k for alpha = +-1)
// the product is formed by integer operations on the bit patterns, so each
// element costs one FP64 addition instead of a multiplication, a conversion
// and a fused multiply-add at GB300's FP64 rate.
__global__ void split_flush_kernel(long long M, int N, const float* __restrict__ P,
                                   const double* __restrict__ mu, const double* __restrict__ nu,
                                   double sc, double* __restrict__ y) {
  if ((N & 3) == 0 && pow2_exp(fabs(sc)) != INT_MIN) {
    const int n4 = N >> 2;
    const double2* nu2 = reinterpret_cast<const double2*>(nu);
    for (long long r = blockIdx.x; r < M; r += gridDim.x) {
      const double s = sc * mu[r];
      const int kr = pow2_exp(fabs(s));
      const float4* pr = reinterpret_cast<const float4*>(P + r * N);
      double2* yr = reinterpret_cast<double2*>(y + r * N);
      for (int c4 = threadIdx.x; c4 < n4; c4 += blockDim.x) {
        const float4 p = __ldcs(pr + c4);
        const double2 na = nu2[2 * c4], nb = nu2[2 * c4 + 1];
        double2 a = yr[2 * c4], b = yr[2 * c4 + 1];
        const int k0 = pow2_exp(na.x), k1 = pow2_exp(na.y), k2 = pow2_exp(nb.x),
                  k3 = pow2_exp(nb.y);
        if (kr != INT_MIN && k0 != INT_MIN && k1 != INT_MIN && k2 != INT_MIN && k3 != INT_MIN) {
          const float sg = s < 0.0 ? -1.f : 1.f;
          a.x += scaled_f2d(sg * p.x, kr + k0);
          a.y += scaled_f2d(sg * p.y, kr + k1);
          b.x += scaled_f2d(sg * p.z, kr + k2);
          b.y += scaled_f2d(sg * p.w, kr + k3);
        } else {
          a.x = fma(s * na.x, (double)p.x, a.x);
          a.y = fma(s * na.y, (double)p.y, a.y);
          b.x = fma(s * nb.x, (double)p.z, b.x);
          b.y = fma(s * nb.y, (double)p.w, b.y);
        }
        yr[2 * c4] = a;
        yr[2 * c4 + 1] = b;
      }
    }
  } else if ((N & 3) == 0) {
    const int n4 = N >> 2;
    const double2* nu2 = reinterpret_cast<const double2*>(nu);
    for (long long r = blockIdx.x; r < M; r += gridDim.x) {
      const double s = sc * mu[r];
      const float4* pr = reinterpret_cast<const float4*>(P + r * N);
      double2* yr = reinterpret_cast<double2*>(y + r * N);
      for (int c4 = threadIdx.x; c4 < n4; c4 += blockDim.x) {
        const float4 p = __ldcs(pr + c4);
        const double2 na = nu2[2 * c4], nb = nu2[2 * c4 + 1];
        double2 a = yr[2 * c4], b = yr[2 * c4 + 1];
        a.x = fma(s * na.x, (double)p.x, a.x);
        a.y = fma(s * na.y, (double)p.y, a.y);
        b.x = fma(s * nb.x, (double)p.z, b.x);
        b.y = fma(s * nb.y, (double)p.w, b.y);
        yr[2 * c4] = a;
        yr[2 * c4 + 1] = b;
      }
    }
  } else {
    for (long long r = blockIdx.x; r < M; r += gridDim.x) {
      const double s = sc * mu[r];
      for (int c = threadIdx.x; c < N; c += blockDim.x)
        y[r * N + c] = fma(s * nu[c], (double)P[r * N + c], y[r * N + c]);
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
  long long grid = M;
  if (grid > 152LL * 16) grid = 152LL * 16;
  if (grid < 1) grid = 1;
  split_flush_kernel<<<(unsigned)grid, 256, 0, st>>>(M, N, P, mu, nu, sc, y);
}

}  // namespace amgt
