// Vector kernels of restarted GMRES: fused multi-dot products and updates for
// classical Gram-Schmidt applied twice (CGS2), linear combinations and
// precision conversions.  Reductions are deterministic: each block writes its
// partial sums to `partials[block][v]` and one block sums them in a fixed
// order.  Arithmetic runs in the vectors' precision; partial sums of FP32
// vectors are FP32 per thread and FP64 across threads.  Every kernel streams
// its vectors four elements at a time with 16-byte accesses (one float4, two
// double2) where all its pointers are 16-byte aligned, and the last n mod 4
// elements (or everything, for unaligned pointers) one at a time.
#include <atomic>
#include <cstdint>
#include <type_traits>

#include "kernels.cuh"

namespace amgt {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxVec = 32;

template <class T>
struct Acc {
  using type = double;
};
template <>
struct Acc<float> {
  using type = float;
};

// four consecutive elements at p (16-byte aligned)
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ bool al16(const void* p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

template <int NV>
__device__ void block_reduce_store(double (&v)[NV], int nvec, double* __restrict__ partials) {
  __shared__ double red[kThreads / 32][kMaxVec];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    if (k >= nvec) break;
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[wid][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < nvec) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
    partials[(long long)blockIdx.x * nvec + threadIdx.x] = s;
  }
}

// out[v] = sum_i V[v][i] * w[i]
template <class T, int NV>
__global__ void __launch_bounds__(kThreads) multidot_kernel(long long n, int nvec,
                                                            const T* const* __restrict__ V,
                                                            const T* __restrict__ w,
                                                            double* __restrict__ partials) {
  using A = typename Acc<T>::type;
  A acc[NV];
  const T* Vk[NV];
  bool vec = al16(w);
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    acc[k] = A(0);
    Vk[k] = k < nvec ? V[k] : w;
    vec = vec && al16(Vk[k]);
  }
  const long long start = blockIdx.x * (long long)kThreads + threadIdx.x;
  const long long stride = (long long)gridDim.x * kThreads;
  long long i0 = 0;
  if (vec) {
    for (long long i = start; i < (n >> 2); i += stride) {
      T wv[4];
      ld4(w + 4 * i, wv);
#pragma unroll
      for (int k = 0; k < NV; ++k)
        if (k < nvec) {
          T vv[4];
          ld4(Vk[k] + 4 * i, vv);
          acc[k] += ((A)vv[0] * (A)wv[0] + (A)vv[1] * (A)wv[1]) +
                    ((A)vv[2] * (A)wv[2] + (A)vv[3] * (A)wv[3]);
        }
    }
    i0 = (n >> 2) << 2;
  }
  for (long long i = i0 + start; i < n; i += stride) {
    const A wi = (A)w[i];
#pragma unroll
    for (int k = 0; k < NV; ++k)
      if (k < nvec) acc[k] += (A)Vk[k][i] * wi;
  }
  double d[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) d[k] = (double)acc[k];
  block_reduce_store<NV>(d, nvec, partials);
}

// w[i] -= sum_v h[v] V[v][i]; then (do_dot == 1) out[v] = sum_i V[v][i] w[i]
// or (do_dot == 2) out[0] = sum_i w[i]^2
template <class T, int NV>
__global__ void __launch_bounds__(kThreads) update_multidot_kernel(
    long long n, int nvec, const T* const* __restrict__ V, const double* __restrict__ h,
    T* __restrict__ w, int do_dot, double* __restrict__ partials) {
  using A = typename Acc<T>::type;
  __shared__ double hs[kMaxVec];
  if (threadIdx.x < nvec) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  A acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = A(0);
  A hA[NV];
  // the 16-byte form keeps 4 NV values of V in registers: up to 8 vectors
  constexpr int KV = NV <= 8 ? NV : 1;
  const T* Vk[KV];
  bool vec = NV <= 8 && al16(w);
#pragma unroll
  for (int k = 0; k < NV; ++k) hA[k] = k < nvec ? (A)hs[k] : A(0);
#pragma unroll
  for (int k = 0; k < KV; ++k) {
    Vk[k] = k < nvec ? V[k] : w;
    vec = vec && al16(Vk[k]);
  }
  const long long start = blockIdx.x * (long long)kThreads + threadIdx.x;
  const long long stride = (long long)gridDim.x * kThreads;
  long long i0 = 0;
  if (vec) {
    for (long long i = start; i < (n >> 2); i += stride) {
      T vk[KV][4], wv[4];
      ld4(w + 4 * i, wv);
      A wa[4] = {(A)wv[0], (A)wv[1], (A)wv[2], (A)wv[3]};
#pragma unroll
      for (int k = 0; k < KV; ++k)
        if (k < nvec) {
          ld4(Vk[k] + 4 * i, vk[k]);
#pragma unroll
          for (int u = 0; u < 4; ++u) wa[u] -= hA[k] * (A)vk[k][u];
        }
      T wn[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) wn[u] = (T)wa[u];
      st4(w + 4 * i, wn);
      if (do_dot == 1) {
#pragma unroll
        for (int k = 0; k < KV; ++k)
          if (k < nvec)
            acc[k] += ((A)vk[k][0] * (A)wn[0] + (A)vk[k][1] * (A)wn[1]) +
                      ((A)vk[k][2] * (A)wn[2] + (A)vk[k][3] * (A)wn[3]);
      } else if (do_dot == 2) {
        acc[0] += ((A)wn[0] * (A)wn[0] + (A)wn[1] * (A)wn[1]) +
                  ((A)wn[2] * (A)wn[2] + (A)wn[3] * (A)wn[3]);
      }
    }
    i0 = (n >> 2) << 2;
  }
  for (long long i = i0 + start; i < n; i += stride) {
    T vk[NV];
    A wi = (A)w[i];
#pragma unroll
    for (int k = 0; k < NV; ++k)
      if (k < nvec) {
        vk[k] = (NV <= 8 ? Vk[k < KV ? k : 0] : V[k])[i];
        wi -= hA[k] * (A)vk[k];
      }
    const T wn = (T)wi;
    w[i] = wn;
    if (do_dot == 1) {
#pragma unroll
      for (int k = 0; k < NV; ++k)
        if (k < nvec) acc[k] += (A)vk[k] * (A)wn;
    } else if (do_dot == 2) {
      acc[0] += (A)wn * (A)wn;
    }
  }
  if (do_dot == 0) return;
  const int nout = do_dot == 1 ? nvec : 1;
  double d[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) d[k] = (double)acc[k];
  block_reduce_store<NV>(d, nout, partials);
}

__global__ void finish_kernel(int nblk, int nvec, const double* __restrict__ partials,
                              double* __restrict__ out) {
  // one warp per output, fixed summation order
  const int lane = threadIdx.x & 31;
  for (int v = threadIdx.x >> 5; v < nvec; v += blockDim.x >> 5) {
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += partials[(long long)b * nvec + v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[v] = s;
  }
}

template <class T>
__global__ void axpby_kernel(long long n, double alpha, const T* __restrict__ x, double beta,
                             T* __restrict__ y) {
  const T a = (T)alpha, bb = (T)beta;
  const long long start = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i0 = 0;
  if (al16(x) && al16(y)) {
    for (long long i = start; i < (n >> 2); i += stride) {
      T xv[4], yv[4];
      ld4(x + 4 * i, xv);
      if (beta != 0.0) ld4(y + 4 * i, yv);
#pragma unroll
      for (int u = 0; u < 4; ++u) yv[u] = beta != 0.0 ? a * xv[u] + bb * yv[u] : a * xv[u];
      st4(y + 4 * i, yv);
    }
    i0 = (n >> 2) << 2;
  }
  for (long long i = i0 + start; i < n; i += stride) {
    T v = a * x[i];
    if (beta != 0.0) v += bb * y[i];
    y[i] = v;
  }
}

template <class T>
__global__ void scale_copy_kernel(long long n, double alpha, const T* __restrict__ x,
                                  T* __restrict__ y) {
  const T a = (T)alpha;
  const long long start = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i0 = 0;
  if (al16(x) && al16(y)) {
    for (long long i = start; i < (n >> 2); i += stride) {
      T v[4];
      ld4(x + 4 * i, v);
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] *= a;
      st4(y + 4 * i, v);
    }
    i0 = (n >> 2) << 2;
  }
  for (long long i = i0 + start; i < n; i += stride) y[i] = a * x[i];
}

template <class Tin, class Tout>
__global__ void convert_kernel(long long n, const Tin* __restrict__ x, Tout* __restrict__ y) {
  const long long start = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i0 = 0;
  if constexpr (sizeof(Tout) >= 4) {
    if (al16(x) && al16(y)) {
      for (long long i = start; i < (n >> 2); i += stride) {
        Tin v[4];
        ld4(x + 4 * i, v);
        Tout o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) o[u] = (Tout)v[u];
        st4(y + 4 * i, o);
      }
      i0 = (n >> 2) << 2;
    }
  }
  for (long long i = i0 + start; i < n; i += stride) y[i] = (Tout)x[i];
}

template <>
__global__ void convert_kernel<float, __nv_bfloat16>(long long n, const float* __restrict__ x,
                                                     __nv_bfloat16* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// x[i] += sum_v y[v] Z[v][i]
template <class T, int NV>
__global__ void __launch_bounds__(kThreads) lincomb_kernel(long long n, int nvec,
                                                           const T* const* __restrict__ Z,
                                                           const double* __restrict__ y,
                                                           T* __restrict__ x) {
  __shared__ T ys[kMaxVec];
  if (threadIdx.x < nvec) ys[threadIdx.x] = (T)y[threadIdx.x];
  __syncthreads();
  const T* Zk[NV];
  bool vec = al16(x);
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    Zk[k] = k < nvec ? Z[k] : x;
    vec = vec && al16(Zk[k]);
  }
  const long long start = blockIdx.x * (long long)kThreads + threadIdx.x;
  const long long stride = (long long)gridDim.x * kThreads;
  long long i0 = 0;
  if (vec) {
    for (long long i = start; i < (n >> 2); i += stride) {
      T v[4];
      ld4(x + 4 * i, v);
#pragma unroll
      for (int k = 0; k < NV; ++k)
        if (k < nvec) {
          T z[4];
          ld4(Zk[k] + 4 * i, z);
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] += ys[k] * z[u];
        }
      st4(x + 4 * i, v);
    }
    i0 = (n >> 2) << 2;
  }
  for (long long i = i0 + start; i < n; i += stride) {
    T v = x[i];
#pragma unroll
    for (int k = 0; k < NV; ++k)
      if (k < nvec) v += ys[k] * Zk[k][i];
    x[i] = v;
  }
}

int grid_1d(long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  if (g > 152LL * 8) g = 152LL * 8;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

int gemv_blocks(long long n) { return grid_1d(n); }

static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// The kernels are instantiated per vector count up to 8 (16 and 32 above):
// where an unused vector slot points at valid memory the compiler may compute
// it and discard the result, which at GB300's FP64 rate made an FP64 norm in
// the 8-slot form 8x slower (36.7 against 4.6 ms for 12.9 GB).
template <class F>
void by_count(int nvec, F f) {
  switch (nvec) {
    case 1: f(std::integral_constant<int, 1>()); break;
    case 2: f(std::integral_constant<int, 2>()); break;
    case 3: f(std::integral_constant<int, 3>()); break;
    case 4: f(std::integral_constant<int, 4>()); break;
    case 5: f(std::integral_constant<int, 5>()); break;
    case 6: f(std::integral_constant<int, 6>()); break;
    case 7: f(std::integral_constant<int, 7>()); break;
    case 8: f(std::integral_constant<int, 8>()); break;
    default:
      if (nvec <= 16) f(std::integral_constant<int, 16>());
      else f(std::integral_constant<int, kMaxVec>());
  }
}

template <class T>
void launch_multidot(long long n, int nvec, const T* const* V, const T* w, double* partials,
                     int nblk, double* out, cudaStream_t st) {
  note_launch(2);
  by_count(nvec, [&](auto nv) {
    multidot_kernel<T, decltype(nv)::value><<<nblk, kThreads, 0, st>>>(n, nvec, V, w, partials);
  });
  finish_kernel<<<1, 1024, 0, st>>>(nblk, nvec, partials, out);
}

template <class T>
void launch_update_multidot(long long n, int nvec, const T* const* V, const double* h, T* w,
                            int do_dot, double* partials, int nblk, double* out,
                            cudaStream_t st) {
  note_launch(do_dot ? 2 : 1);
  by_count(nvec, [&](auto nv) {
    update_multidot_kernel<T, decltype(nv)::value><<<nblk, kThreads, 0, st>>>(n, nvec, V, h, w,
                                                                              do_dot, partials);
  });
  if (do_dot) finish_kernel<<<1, 1024, 0, st>>>(nblk, do_dot == 1 ? nvec : 1, partials, out);
}

template <class T>
void launch_axpby(long long n, double alpha, const T* x, double beta, T* y, cudaStream_t st) {
  note_launch();
  axpby_kernel<T><<<grid_1d(n), kThreads, 0, st>>>(n, alpha, x, beta, y);
}

template <class T>
void launch_scale_copy(long long n, double alpha, const T* x, T* y, cudaStream_t st) {
  note_launch();
  scale_copy_kernel<T><<<grid_1d(n), kThreads, 0, st>>>(n, alpha, x, y);
}

template <class Tin, class Tout>
void launch_convert(long long n, const Tin* x, Tout* y, cudaStream_t st) {
  note_launch();
  convert_kernel<Tin, Tout><<<grid_1d(n), kThreads, 0, st>>>(n, x, y);
}

// Phi[r][k] *= fdeg[fid[r / s]][k]: moments scaled by each cell's moment shape
template <class T>
__global__ void scale_moments_kernel(long long rows, int s, int nmom, const int* __restrict__ fid,
                                     const T* __restrict__ fdeg, T* __restrict__ Phi) {
  const long long total = rows * nmom;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / nmom;
    const int k = (int)(i - r * nmom);
    Phi[i] *= fdeg[(size_t)fid[r / s] * nmom + k];
  }
}

template <class T>
void launch_scale_moments(long long rows, int s, int nmom, const int* fid, const T* fdeg, T* Phi,
                          cudaStream_t st) {
  note_launch();
  scale_moments_kernel<T><<<grid_1d(rows * nmom), kThreads, 0, st>>>(rows, s, nmom, fid, fdeg,
                                                                      Phi);
}

template <class T>
void launch_lincomb(long long n, int nvec, const T* const* Z, const double* y, T* x,
                    cudaStream_t st) {
  note_launch();
  by_count(nvec, [&](auto nv) {
    lincomb_kernel<T, decltype(nv)::value><<<grid_1d(n), kThreads, 0, st>>>(n, nvec, Z, y, x);
  });
}

#define AMGT_INST(T)                                                                          \
  template void launch_multidot<T>(long long, int, const T* const*, const T*, double*, int,  \
                                   double*, cudaStream_t);                                   \
  template void launch_update_multidot<T>(long long, int, const T* const*, const double*, T*, \
                                          int, double*, int, double*, cudaStream_t);          \
  template void launch_axpby<T>(long long, double, const T*, double, T*, cudaStream_t);      \
  template void launch_scale_copy<T>(long long, double, const T*, T*, cudaStream_t);         \
  template void launch_lincomb<T>(long long, int, const T* const*, const double*, T*,        \
                                  cudaStream_t);                                             \
  template void launch_scale_moments<T>(long long, int, int, const int*, const T*, T*,       \
                                        cudaStream_t);
AMGT_INST(double)
AMGT_INST(float)
#undef AMGT_INST
template void launch_convert<double, float>(long long, const double*, float*, cudaStream_t);
template void launch_convert<float, double>(long long, const float*, double*, cudaStream_t);
template void launch_convert<float, __nv_bfloat16>(long long, const float*, __nv_bfloat16*,
                                                   cudaStream_t);
template void launch_convert<double, __nv_bfloat16>(long long, const double*, __nv_bfloat16*,
                                                    cudaStream_t);

}  // namespace amgt
