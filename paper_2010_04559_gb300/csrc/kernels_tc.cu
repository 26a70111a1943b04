// BF16 tensor-core contraction of the scatter source (Sec. 4.2) on the fifth-
// generation tensor cores (tcgen05, sm_103a):
//
//   Y[M][N] = (sigma_s N (x) I) X S  (+ beta Y + add)
//
// The per-cell factor sigma_s N (a mixing of the s rows of one cell) commutes
// with the right-multiplication by the angular matrix S, so it is applied in
// the FP32 -> BF16 operand pass (`tc_prep_kernel`) and the GEMM epilogue only
// adds.  GEMM: a persistent kernel, one CTA per SM walking the 128 x 256
// output tiles; A = X (row-major, K-major) and B = S^T = S (symmetric,
// K-major) are loaded by TMA with the 128-byte swizzle into a 4-stage
// shared-memory ring guarded by mbarriers; one thread issues tcgen05.mma
// (M=128, N=256, K=16, BF16 inputs, FP32 accumulation) into one of two
// 256-column tensor-memory accumulators, so that eight epilogue warps drain
// tile i (tcgen05.ld, FP32 stores) while the MMAs of tile i+1 run.  Every
// wait is bounded: after 2 s the kernel records an error code, lets its
// in-flight copies and MMAs finish (bounded again), releases its tensor
// memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <mutex>

#include "kernels.cuh"

namespace amgt {

namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_WARPS = 8;                      // two per accumulator lane quarter
constexpr int TC_THREADS = 64 + 32 * EPI_WARPS;  // producer warp, MMA warp, epilogue
constexpr uint32_t TMEM_COLS = 2 * BN;            // two accumulators
constexpr unsigned long long kWaitNs = 2000000000ULL;
constexpr size_t kSmemBytes = (size_t)STAGES * STAGE_BYTES + 1024 + 256;

// instruction descriptor: D f32, A/B bf16 (F16 = false) or f16 (F16 = true),
// both K-major, N >> 3, M >> 4
template <bool F16>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | (F16 ? 0u : (1u << 7) | (1u << 10)) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

struct TcArgs {
  int M, N, K;
  float* C;
  const float* add;
  float beta;
  const float* rs;  // optional per-row scale of the product (null: 1)
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false after kWaitNs or when another role has aborted
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  const unsigned long long t0 = now_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63) {
      if (*abort_flag) return false;
      if (now_ns() - t0 > kWaitNs) return false;
    }
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}
// shared-memory matrix descriptor, K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}
__device__ __forceinline__ void umma_16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t id, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(id), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Output tile t -> (row, column) tile origin.  Tiles run in groups of kGroupN
// column tiles, the column tile fastest within a group: the CTAs working at
// the same time share the k-chunks of ~152 / kGroupN row tiles of A and of
// kGroupN column tiles of B, so both stay in L2 while they are read
// (with every column tile in one group, all of B streams past each wave of
// row tiles and is re-read from DRAM).
constexpr int kGroupN = 8;
__device__ __forceinline__ void tile_origin(int t, int m_tiles, int n_tiles, int& m0, int& n0) {
  const int gsz = kGroupN * m_tiles;
  const int grp = t / gsz, r = t - grp * gsz;
  const int gw = min(kGroupN, n_tiles - grp * kGroupN);
  m0 = (r / gw) * BM;
  n0 = (grp * kGroupN + r % gw) * BN;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// one accumulator chunk (32 columns of this thread's row) to global memory
__device__ __forceinline__ void store_chunk(float* out, const float* ad, const float4 (&a4)[8],
                                            const uint32_t (&v)[32], float beta, float rsc,
                                            bool vec, int ncols) {
  if (vec) {
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
      float4 o = make_float4(rsc * __uint_as_float(v[j]), rsc * __uint_as_float(v[j + 1]),
                             rsc * __uint_as_float(v[j + 2]), rsc * __uint_as_float(v[j + 3]));
      if (beta != 0.0f) {
        const float4 b = *reinterpret_cast<const float4*>(out + j);
        o.x += beta * b.x;
        o.y += beta * b.y;
        o.z += beta * b.z;
        o.w += beta * b.w;
      }
      if (ad) {
        o.x += a4[j / 4].x;
        o.y += a4[j / 4].y;
        o.z += a4[j / 4].z;
        o.w += a4[j / 4].w;
      }
      __stcs(reinterpret_cast<float4*>(out + j), o);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) {  // static register indices
      if (j < ncols) {
        float o = rsc * __uint_as_float(v[j]);
        if (beta != 0.0f) o += beta * out[j];
        if (ad) o += ad[j];
        out[j] = o;
      }
    }
  }
}

template <bool F16>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                 const __grid_constant__ CUtensorMap tmB,
                                                                 TcArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;  // [2] accumulator ready (MMA -> epilogue)
  uint64_t* acce = accf + 2;        // [2] accumulator drained (epilogue -> MMA)
  uint64_t* done = acce + 2;        // every issued MMA complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tiles = (args.N + BN - 1) / BN;
  const int m_tiles = (args.M + BM - 1) / BM;
  const int total = n_tiles * m_tiles;
  const int kiters = (args.K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], EPI_WARPS);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer: the ring runs continuously across this CTA's tiles
      int g = 0;
      for (int t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x) {
        int m0, n0;
        tile_origin(t, m_tiles, n_tiles, m0, n0);
        for (int k = 0; k < kiters; ++k, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
            *abort_flag = 1;
            atomicExch(args.err, 1);
            break;
          }
          uint8_t* sa = smem + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          tma_load_2d(sa, &tmA, &full[s], k * BK, m0);
          tma_load_2d(sa + A_BYTES, &tmB, &full[s], k * BK, n0);
        }
      }
      if (*abort_flag) {
        // let the copies already issued land before the CTA exits
        for (int k = g > STAGES ? g - STAGES : 0; k < g; ++k) {
          volatile int never = 0;
          mbar_wait(&full[k % STAGES], (uint32_t)(k / STAGES) & 1u, &never);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      int g = 0, i = 0;
      for (int t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x, ++i) {
        const int buf = i & 1;
        const uint32_t use = (uint32_t)(i >> 1) & 1u;
        if (!mbar_wait(&acce[buf], use ^ 1u, abort_flag)) {
          *abort_flag = 1;
          atomicExch(args.err, 2);
          break;
        }
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(buf * BN);
        bool ok = true;
        for (int k = 0; k < kiters; ++k, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
          if (!mbar_wait(&full[s], ph, abort_flag)) {
            *abort_flag = 1;
            atomicExch(args.err, 2);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
          const uint64_t adesc = sw128_desc(sa);
          const uint64_t bdesc = sw128_desc(sa + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            umma_16(dt, adesc + 2ull * kk, bdesc + 2ull * kk, idesc<F16>(), (k | kk) != 0 ? 1u : 0u);
          umma_commit(&empty[s]);
        }
        if (!ok) break;
        umma_commit(&accf[buf]);
      }
      // completion of every MMA issued above (also on abort)
      umma_commit(done);
      volatile int never = 0;
      if (!mbar_wait(done, 0, &never)) atomicExch(args.err, 2);
    }
  } else {
    // epilogue: warp w reads accumulator lanes 32 (w % 4) .. +31 (its rows) and
    // one half of the columns
    const int q = warp & 3, h = (warp - 2) >> 2;
    const bool vec = (args.N & 3) == 0;
    int i = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++i) {
      int m0, n0;
      tile_origin(t, m_tiles, n_tiles, m0, n0);
      const int buf = i & 1;
      const uint32_t use = (uint32_t)(i >> 1) & 1u;
      bool ok = mbar_wait(&accf[buf], use, abort_flag);
      ok = __all_sync(0xffffffffu, ok && !*abort_flag);  // tcgen05.ld is warp-collective
      if (!ok) {
        *abort_flag = 1;
        atomicExch(args.err, 3);
        break;
      }
      tc_fence_after();
      const int row = m0 + q * 32 + lane;
      const bool rowok = row < args.M;
      const int cbase = n0 + h * (BN / 2);
      const float* adrow = args.add ? args.add + (long long)row * args.N : nullptr;
      // the scale is exactly 1 without a row-scale vector
      const float rsc = (args.rs && rowok) ? args.rs[row] : 1.0f;
      // add for chunk c+1 is loaded while chunk c is stored (two register sets)
      float4 aA[8], aB[8];
      auto load_add = [&](int c, float4(&dst)[8]) {
        const int col0 = cbase + c * 32;
        if (adrow && rowok && vec && col0 + 32 <= args.N) {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            dst[j] = __ldcs(reinterpret_cast<const float4*>(adrow + col0) + j);
        }
      };
      auto drain = [&](int c, const float4(&cur)[8]) {
        const int col0 = cbase + c * 32;
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + h * (BN / 2) + c * 32), v);
        if (rowok && col0 < args.N) {
          const int ncols = min(32, args.N - col0);
          store_chunk(args.C + (long long)row * args.N + col0, adrow ? adrow + col0 : nullptr, cur,
                      v, args.beta, rsc, vec && ncols == 32, ncols);
        }
      };
      static_assert(BN / 64 == 4, "four 32-column chunks per epilogue warp");
      load_add(0, aA);
      load_add(1, aB);
      drain(0, aA);
      load_add(2, aA);
      drain(1, aB);
      load_add(3, aB);
      drain(2, aA);
      drain(3, aB);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// Xb[c*s+l][j] = bf16(alpha * sig[c] * sum_i N[l][i] x[c*s+i][j])
template <int S>
__global__ void tc_prep_kernel(long long ncell, int n, const float* __restrict__ x,
                               const float* __restrict__ sig, const float* __restrict__ Nm,
                               float alpha, __nv_bfloat16* __restrict__ xb) {
  const long long total = ncell * (long long)n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = idx / n;
    const int j = (int)(idx - c * n);
    float v[S];
#pragma unroll
    for (int i = 0; i < S; ++i) v[i] = x[(c * S + i) * n + j];
    const float f = alpha * sig[c];
#pragma unroll
    for (int l = 0; l < S; ++l) {
      float a = 0.f;
#pragma unroll
      for (int i = 0; i < S; ++i) a += Nm[l * S + i] * v[i];
      xb[(c * S + l) * n + j] = __float2bfloat16_rn(f * a);
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool encode_kmajor(CUtensorMap* m, const void* ptr, int rows, int K, int box_rows, bool f16) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
            const_cast<void*>(ptr), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool tc_available() {
  cudaFuncAttributes a;
  return cudaFuncGetAttributes(&a, tc_gemm_kernel<false>) == cudaSuccess &&
         cudaFuncGetAttributes(&a, tc_gemm_kernel<true>) == cudaSuccess && encode_fn() != nullptr;
}

void launch_tc_prep(long long ncell, int s, int n, const float* x, const float* sig,
                    const float* Nm, float alpha, __nv_bfloat16* xb, cudaStream_t st) {
  note_launch();
  const long long total = ncell * (long long)n;
  long long grid = (total + 255) / 256;
  if (grid > 152LL * 16) grid = 152LL * 16;
  if (s == 4)
    tc_prep_kernel<4><<<(int)grid, 256, 0, st>>>(ncell, n, x, sig, Nm, alpha, xb);
  else
    tc_prep_kernel<8><<<(int)grid, 256, 0, st>>>(ncell, n, x, sig, Nm, alpha, xb);
}

// C = rs (A B) (+ beta C + add): A [M][K] and Bt [N][K] (B^T) both bf16 or
// both f16, C/add [M][N] f32, rs [M] f32 or null
int launch_tc_gemm_ex(int M, int N, int K, const void* A, const void* Bt, bool f16, float* C,
                      const float* add, float beta, const float* rs, int* err, cudaStream_t st) {
  if (M <= 0 || N < 16 || K < BK || (K % 8) != 0) return -1;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Bt)) & 15) return -1;
  CUtensorMap ta, tb;
  if (!encode_kmajor(&ta, A, M, K, BM, f16) || !encode_kmajor(&tb, Bt, N, K, BN, f16)) return -2;
  // per launch: the attribute and the SM count belong to the current device
  if (allow_max_smem(f16 ? tc_gemm_kernel<true> : tc_gemm_kernel<false>) != cudaSuccess)
    return -3;
  TcArgs args{M, N, K, C, add, beta, rs, err};
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (nsm <= 0) nsm = 1;
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  const int grid = tiles < nsm ? tiles : nsm;
  note_launch();
  if (f16)
    tc_gemm_kernel<true><<<grid, TC_THREADS, kSmemBytes, st>>>(ta, tb, args);
  else
    tc_gemm_kernel<false><<<grid, TC_THREADS, kSmemBytes, st>>>(ta, tb, args);
  return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

int launch_tc_gemm(int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* Bt, float* C,
                   const float* add, float beta, int* err, cudaStream_t st) {
  return launch_tc_gemm_ex(M, N, K, A, Bt, false, C, add, beta, nullptr, err, st);
}

}  // namespace amgt
