// FP32-accurate scatter contraction (Sec. 4.2) on FP16 tensor cores.
//
//   Y = (sigma_s N (x) I) X S,  X and Y FP32
//
// Each row z of the cell-mixed operand sigma_s N x is scaled by a power of two
// so that its largest entry lies in [2^14, 2^15), and cut into a high and a
// low FP16 part, z 2^e = hi + lo + O(2^-22 max|z| 2^e); S_f is cut the same
// way with one power-of-two scale.  The three products hi S_hi + lo S_hi +
// hi S_lo (the lo S_lo term lies ~2^-22 below the result) run as ONE tcgen05
// GEMM over the concatenated inner dimension 3K, operands
//
//   A = [hi | lo | hi]   (rows of z, K-major)      Bt = [S_hi | S_hi | S_lo]
//
// with exact FP16 x FP16 products summed in FP32, and the epilogue multiplies
// each row by its inverse scale.  The relative error is ~2^-21, that of an
// FP32 contraction of this length, at three times the BF16 GEMM's work.
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>

#include "kernels.cuh"

namespace amgt {

namespace {

constexpr int kPrepThreads = 256;

// rows r = c S + l of z = alpha sig[c] (N x_c)[l], scaled per row by a power
// of two; out row r = [hi | lo | hi] (3n halves), rs[r] = the inverse scale
// times sinv (the inverse scale of S)
template <int S>
__global__ void __launch_bounds__(kPrepThreads) tc3_prep_kernel(
    long long ncell, int n, const float* __restrict__ x, const float* __restrict__ sig,
    const float* __restrict__ Nm, float alpha, float sinv, __half* __restrict__ out,
    float* __restrict__ rs) {
  __shared__ float red[kPrepThreads / 32][S];
  __shared__ float scl[S];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float nm[S * S];
#pragma unroll
  for (int i = 0; i < S * S; ++i) nm[i] = Nm[i];
  for (long long c = blockIdx.x; c < ncell; c += gridDim.x) {
    const float f = alpha * sig[c];
    const float* xc = x + c * S * (long long)n;
    float mx[S];
#pragma unroll
    for (int l = 0; l < S; ++l) mx[l] = 0.f;
    for (int j = 2 * threadIdx.x; j < n; j += 2 * kPrepThreads) {
      float2 v[S];
#pragma unroll
      for (int i = 0; i < S; ++i) v[i] = *reinterpret_cast<const float2*>(xc + (long long)i * n + j);
#pragma unroll
      for (int l = 0; l < S; ++l) {
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int i = 0; i < S; ++i) {
          a0 += nm[l * S + i] * v[i].x;
          a1 += nm[l * S + i] * v[i].y;
        }
        mx[l] = fmaxf(mx[l], fmaxf(fabsf(f * a0), fabsf(f * a1)));
      }
    }
#pragma unroll
    for (int l = 0; l < S; ++l) {
      float m = mx[l];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) red[warp][l] = m;
    }
    __syncthreads();
    if (threadIdx.x < S) {
      const int l = threadIdx.x;
      float m = 0.f;
      for (int w = 0; w < kPrepThreads / 32; ++w) m = fmaxf(m, red[w][l]);
      float sc = 0.f, inv = 0.f;
      if (m > 0.f && m <= 3.0e38f) {
        const int e = ilogbf(m);  // m in [2^e, 2^(e+1))
        sc = ldexpf(1.f, 14 - e);
        inv = ldexpf(1.f, e - 14) * sinv;
      }
      scl[l] = sc;
      rs[c * S + l] = inv;
    }
    __syncthreads();
    for (int j = 2 * threadIdx.x; j < n; j += 2 * kPrepThreads) {
      float2 v[S];
#pragma unroll
      for (int i = 0; i < S; ++i) v[i] = *reinterpret_cast<const float2*>(xc + (long long)i * n + j);
#pragma unroll
      for (int l = 0; l < S; ++l) {
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int i = 0; i < S; ++i) {
          a0 += nm[l * S + i] * v[i].x;
          a1 += nm[l * S + i] * v[i].y;
        }
        const float t0 = (f * a0) * scl[l], t1 = (f * a1) * scl[l];
        const __half h0 = __float2half_rn(t0), h1 = __float2half_rn(t1);
        // t - hi is exact in FP32 (hi is t rounded to 11 significant bits)
        const __half l0 = __float2half_rn(t0 - __half2float(h0));
        const __half l1 = __float2half_rn(t1 - __half2float(h1));
        __half* row = out + (c * S + l) * 3LL * n;
        const __half2 hh = __halves2half2(h0, h1), ll = __halves2half2(l0, l1);
        *reinterpret_cast<__half2*>(row + j) = hh;
        *reinterpret_cast<__half2*>(row + n + j) = ll;
        *reinterpret_cast<__half2*>(row + 2 * n + j) = hh;
      }
    }
    __syncthreads();  // red/scl are reused by the next cell
  }
}

// largest |S| as the bit pattern of a non-negative double (ordered as integers)
__global__ void tc3_absmax_kernel(long long total, const double* __restrict__ Sf,
                                  unsigned long long* __restrict__ mx) {
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(Sf[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

// Bt row c = [S_hi(c, :) | S_hi(c, :) | S_lo(c, :)] of sc S (S symmetric)
__global__ void tc3_split_sf_kernel(int n, const double* __restrict__ Sf, double sc,
                                    __half* __restrict__ Bt) {
  const long long total = (long long)n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / n;
    const int k = (int)(i - c * n);
    const double t = Sf[i] * sc;
    const __half hi = __double2half(t);
    const __half lo = __double2half(t - (double)__half2float(hi));
    __half* row = Bt + c * 3LL * n;
    row[k] = hi;
    row[n + k] = hi;
    row[2 * n + k] = lo;
  }
}

}  // namespace

void launch_tc3_prep(long long ncell, int s, int n, const float* x, const float* sig,
                     const float* Nm, float alpha, float sinv, __half* out, float* rs,
                     cudaStream_t st) {
  note_launch();
  long long grid = ncell;
  if (grid > 152LL * 8) grid = 152LL * 8;
  if (grid < 1) grid = 1;
  if (s == 4)
    tc3_prep_kernel<4><<<(int)grid, kPrepThreads, 0, st>>>(ncell, n, x, sig, Nm, alpha, sinv, out, rs);
  else
    tc3_prep_kernel<8><<<(int)grid, kPrepThreads, 0, st>>>(ncell, n, x, sig, Nm, alpha, sinv, out, rs);
}

cudaError_t tc3_split_sf(int n, const double* Sf, unsigned long long* dmax, __half* Bt,
                         double* sinv_out, cudaStream_t st) {
  const long long total = (long long)n * n;
  cudaError_t e = cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  long long grid = (total + 255) / 256;
  if (grid > 152LL * 8) grid = 152LL * 8;
  note_launch();
  tc3_absmax_kernel<<<(int)grid, 256, 0, st>>>(total, Sf, dmax);
  unsigned long long bits = 0;
  e = cudaMemcpyAsync(&bits, dmax, sizeof(bits), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  double m;
  static_assert(sizeof(m) == sizeof(bits), "double is 64 bits");
  memcpy(&m, &bits, sizeof(m));
  double sc = 0.0;
  *sinv_out = 0.0;
  if (m > 0.0) {
    const int ex = std::ilogb(m);
    sc = std::ldexp(1.0, 14 - ex);
    *sinv_out = std::ldexp(1.0, ex - 14);
  }
  note_launch();
  tc3_split_sf_kernel<<<(int)grid, 256, 0, st>>>(n, Sf, sc, Bt);
  return cudaGetLastError();
}

}  // namespace amgt
