// Small device helpers shared by the coarse Gauss-Seidel kernels (Sec. 4.2):
// face-node indexing of Q1 cells, padded shared-memory strides, 16-byte dot
// products and the global timer used by bounded waits.
#pragma once
#include <cuda_runtime.h>

namespace amgt {
namespace gsx {

// Q1 node numbering: bit `axis` of a node index is its side along that axis.
// fnode inserts `bit` at position `axis` into a face-node index j (the node
// index with that bit removed); fcompress removes bit `axis` from node l.
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

// vector of 16 bytes of T and its dot product with another
template <class T>
struct V16;
template <>
struct V16<float> {
  static constexpr int n = 4;
  __device__ static float dot(const float* a, const float* b) {
    const float4 x = *reinterpret_cast<const float4*>(a);
    const float4 y = *reinterpret_cast<const float4*>(b);
    return x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
  }
};
template <>
struct V16<double> {
  static constexpr int n = 2;
  __device__ static double dot(const double* a, const double* b) {
    const double2 x = *reinterpret_cast<const double2*>(a);
    const double2 y = *reinterpret_cast<const double2*>(b);
    return x.x * y.x + x.y * y.y;
  }
};

// padded row strides (in elements of T) that spread 16-byte accesses of
// consecutive rows over distinct bank groups: an odd number of 16-byte units
template <class T>
__host__ __device__ inline int pad16(int n) {
  const int vw = 16 / (int)sizeof(T);
  int p = ((n + vw - 1) / vw) * vw;
  if (((p / vw) & 1) == 0) p += vw;
  return p;
}
// n elements of size esz rounded up to whole 16-byte units
__host__ __device__ inline size_t round16(size_t elems, size_t esz) {
  const size_t vw = 16 / esz;
  return ((elems + vw - 1) / vw) * vw;
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace gsx
}  // namespace amgt
