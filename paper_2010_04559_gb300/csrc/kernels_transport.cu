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
#include <cstdint>
#include <type_traits>

#include "gs_common.cuh"
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

// Double-float numbers: a value is hi + lo with two FP32 parts (about 44
// significant bits), added and multiplied with error-free transformations --
// Knuth's two-sum, the fast two-sum for |a| >= |b|, and the exact product of
// two floats from one FMA (Dekker's product written with fmaf) -- following
// the double-float arithmetic of Dekker (1971).  Used where an FP64 result is
// needed to ~1e-13 and GB300's FP32 rate (64x its FP64 rate) pays for the
// ~10 FP32 operations per multiply-add.
struct DF {
  float hi, lo;
  __device__ __forceinline__ DF() : hi(0.f), lo(0.f) {}
  __device__ __forceinline__ DF(int v) : hi((float)v), lo(0.f) {}
  __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit DF(double v) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  }
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return DF(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return DF(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ DF operator+(const DF& a, const DF& b) {
  DF s = df_two_sum(a.hi, b.hi);
  const float t = __fadd_rn(a.lo, b.lo);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, t));
}
__device__ __forceinline__ DF operator-(const DF& a) { return DF(-a.hi, -a.lo); }
__device__ __forceinline__ DF operator*(const DF& a, const DF& b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ DF& operator+=(DF& a, const DF& b) {
  a = a + b;
  return a;
}

// An FP64 value as double-float by integer operations alone (FP64 conversions
// run at the FP64 rate): hi keeps the leading 24 bits of the significand
// (truncated), lo the remaining 29 bits rounded to 24, so hi + lo is the
// value to a relative 2^-47.  Values outside [2^-74, 2^128) and zero take the
// conversion path.
__device__ __forceinline__ DF df_split(double v) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((bits >> 52) & 0x7ffULL) - 1023;
  if (e < -74 || e > 127) {
    if ((bits << 1) == 0ULL) return DF(0.f, 0.f);
    const float h = (float)v;
    return DF(h, (float)(v - (double)h));
  }
  const unsigned sgn = (unsigned)(bits >> 32) & 0x80000000u;
  const float hi =
      __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | (unsigned)((bits >> 29) & 0x7fffffULL));
  const float lo = __fmul_rn(__uint2float_rn((unsigned)(bits & 0x1fffffffULL)),
                             __uint_as_float((unsigned)(e - 52 + 127) << 23));
  return DF(hi, sgn ? -lo : lo);
}
// a float as FP64, exactly, by integer operations (zero and normal floats;
// subnormals, infinities and NaN by conversion)
__device__ __forceinline__ double df_f2d(float f) {
  const unsigned u = __float_as_uint(f);
  if ((u & 0x7fffffffu) == 0u) return 0.0;
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex == 0u || ex == 0xffu) return (double)f;
  return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                          ((unsigned long long)(ex + 896u) << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}
__device__ __forceinline__ double df_to_double(const DF& v) { return df_f2d(v.hi) + df_f2d(v.lo); }

// A dot-product accumulator in the style of Ogita, Rump and Oishi's Dot2
// (2005): the running sum s collects the leading products through two-sum,
// c the exact product errors, the two-sum errors and the cross terms
// hi lo + lo hi in plain FP32 (all ~2^-24 of the sum or smaller).
struct DFAcc {
  float s = 0.f, c = 0.f;
};
__device__ __forceinline__ void df_fma(DFAcc& a, const DF& x, const DF& y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float pe = __fmaf_rn(x.hi, y.hi, -p);
  const float s = __fadd_rn(a.s, p);
  const float bb = __fsub_rn(s, a.s);
  const float se = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  a.s = s;
  a.c = __fadd_rn(a.c, __fadd_rn(__fadd_rn(se, pe), __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi))));
}
__device__ __forceinline__ DF df_val(const DFAcc& a) { return df_two_sum(a.s, a.c); }

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

// ---------------------------------------------------------------------------
// 3D sweep over every direction and patch at once.  In rotated coordinates
// (each direction's axes flipped so that it sweeps from the origin) the
// wavefront levels w = jx + jy + jz are the same for all directions, so one
// cooperative launch walks the levels with a bounded grid barrier between
// them and, within a level, hands out the (cell, patch) items of every
// direction to warps: the patch fixes the direction and so the cell's flips.
// A warp solves one item: lane r = l A + m (r < S A) forms its entry of the
// right-hand side (b minus the upwind faces' coupling) and then its entry of
// the block solve, row r of the block inverse (read as 16-byte chunks) times
// the right-hand side gathered by shuffles.  The level kernel below runs one
// block per (direction, patch group) and leaves most of the GPU idle.
constexpr int kSweep3Threads = 512;

__device__ __forceinline__ void grid_sync_bounded(unsigned* bar, unsigned nblocks, unsigned& gen,
                                                  int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == nblocks) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicExch(bar + 1, gen + 1u);
    } else {
      const unsigned long long t0 = gsx::now_ns();
      unsigned it = 0;
      while (*vgen == gen) {
        if ((++it & 255u) == 0) {
          if (*reinterpret_cast<volatile int*>(err) != 0) break;
          if (gsx::now_ns() - t0 > 2000000000ULL) {
            atomicExch(err, 8);  // a grid barrier of the 3D sweep gave up
            break;
          }
        }
      }
    }
    __threadfence();
  }
  gen += 1u;
  __syncthreads();
}

template <class T, int A>
__global__ void __launch_bounds__(kSweep3Threads) sweep3d_grid_kernel(
    Geom g, LevelDev<T> t, CellData cd, Schedule sc, const T* __restrict__ b,
    T* __restrict__ psi, unsigned* __restrict__ gbar, int* __restrict__ err) {
  constexpr int S = 8;
  constexpr int SA = S * A;
  const int lane = threadIdx.x & 31;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  const int P = g.P, nadof = g.nadof;
  const bool act = lane < SA;
  const int r = act ? lane : 0;
  const int l = r / A, m = r - (r / A) * A;
  const int stride[3] = {1, g.nx, g.nx * g.ny};
  unsigned gen = 0;
  for (int w = 0; w < sc.nlev; ++w) {
    const int beg = sc.level_off[w];
    const long long items = (long long)(sc.level_off[w + 1] - beg) * P;
    for (long long it = wid; it < items; it += nwarp) {
      const int k = (int)(it / P);
      const int q = (int)(it - (long long)k * P);
      int neg[3];
      dir_bits<3>(t.pdir[q], neg);
      const int packed = sc.cells[beg + k];
      const int jj[3] = {packed & 2047, (packed >> 11) & 2047, packed >> 22};
      const int ix = neg[0] ? g.nx - 1 - jj[0] : jj[0];
      const int iy = neg[1] ? g.ny - 1 - jj[1] : jj[1];
      const int iz = neg[2] ? g.nz - 1 - jj[2] : jj[2];
      const int c = ix + g.nx * (iy + g.ny * iz);
      T rhs = T(0);
      if (act) {
        rhs = b[((long long)c * S + l) * nadof + q * A + m];
        // upwind faces: the neighbour's trace on the shared face
#pragma unroll
        for (int xi = 0; xi < 3; ++xi) {
          const int own = neg[xi];
          if (jj[xi] == 0 || ((l >> xi) & 1) != own) continue;
          const int cn = c + (own ? stride[xi] : -stride[xi]);
          const T* An = t.Aax + ((size_t)q * 3 + xi) * A * A + m * A;
          const T* pn = psi + (long long)cn * S * nadof + q * A;
          const int jp = gsx::fcompress(l, xi);
          T acc = T(0);
#pragma unroll
          for (int j = 0; j < S / 2; ++j) {
            const int i = gsx::fnode(j, xi, 1 - own);
            T sacc = T(0);
#pragma unroll
            for (int d = 0; d < A; ++d) sacc += An[d] * __ldcg(pn + (long long)i * nadof + d);
            acc += T(g.facemass[xi][jp][j]) * sacc;
          }
          rhs -= (own ? T(1) : T(-1)) * acc;
        }
      }
      // x_r = sum_cc Kinv[r][cc] rhs_cc
      const T* Ki = t.Kinv + ((size_t)cd.mat[c] * P + q) * SA * SA + (size_t)r * SA;
      T x = T(0);
      constexpr int VW = 16 / (int)sizeof(T);
#pragma unroll
      for (int cc = 0; cc < SA; cc += VW) {
        T kv[VW];
        if constexpr (sizeof(T) == 4 && SA % 4 == 0) {
          const float4 v = *reinterpret_cast<const float4*>(Ki + cc);
          kv[0] = v.x; kv[1] = v.y; kv[2] = v.z; kv[3] = v.w;
        } else if constexpr (sizeof(T) == 8 && SA % 2 == 0) {
          const double2 v = *reinterpret_cast<const double2*>(Ki + cc);
          kv[0] = v.x; kv[1] = v.y;
        } else {
#pragma unroll
          for (int u = 0; u < VW; ++u) kv[u] = cc + u < SA ? Ki[cc + u] : T(0);
        }
#pragma unroll
        for (int u = 0; u < VW; ++u) {
          const T ru = __shfl_sync(0xffffffffu, rhs, (cc + u) < SA ? cc + u : 0);
          if (cc + u < SA) x += kv[u] * ru;
        }
      }
      if (act) psi[((long long)c * S + l) * nadof + q * A + m] = x;
    }
    // the next level reads this level's outputs (other warps, other blocks)
    if (w + 1 < sc.nlev) grid_sync_bounded(gbar, gridDim.x, gen, err);
  }
}

// ---------------------------------------------------------------------------
// 2D sweep, row-pipelined.  For one direction and a group of nq patches, thread
// (jy, p) owns rotated row jy and patch p and visits its row's cells
// jx = 0..nx-1 at wavefront levels w = jx + jy.  The x-upwind values are the
// thread's own previous output (registers); the y-upwind values come from
// row jy-1 through a double-buffered shared row buffer; b is staged NST levels
// ahead with cp.async; the block inverses of the group sit in shared memory.
__device__ __forceinline__ void cp_async_bytes(void* smem, const void* gmem, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <class T, int A, int NST, int UMAX>
__global__ void __launch_bounds__(512) sweep2d_rows_kernel(Geom g, LevelDev<T> t, CellData cd,
                                                            Schedule sc, const T* __restrict__ b,
                                                            T* __restrict__ psi, int G, int nmat_s,
                                                            int chunk) {
  constexpr int S = 4;
  constexpr int SA = S * A;
  constexpr int KST = SA * SA + 16 / sizeof(T);  // padded inverse stride (bank spread)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int task = blockIdx.x;
  const int d = sc.task_dir[task], q0 = sc.task_q0[task], nq = sc.task_nq[task];
  const int negx = (d >> 1) & 1, negy = d & 1;
  const int nx = g.nx, ny = g.ny, nadof = g.nadof;
  const int seg = nq * A;                 // elements per (cell, node) row segment
  const int segp = G * A;                 // padded segment in shared memory
  T* stage = reinterpret_cast<T*>(smem_raw);                     // [NST][ny][S][segp]
  T* yface = stage + (size_t)NST * ny * S * segp;                // [2][ny][G][2][A]
  T* kin = yface + (size_t)2 * ny * G * 2 * A;                   // [nmat_s][G][KST]
  const int tid = threadIdx.x;
  const int p = tid % G, jy = tid / G;
  const bool mine = jy < ny && p < nq;
  const int q = q0 + p;
  // inverses of this group into shared memory
  for (int i = tid; i < nmat_s * nq * SA * SA; i += blockDim.x) {
    const int mt = i / (nq * SA * SA);
    const int rem = i - mt * nq * SA * SA;
    const int pp = rem / (SA * SA), e = rem - pp * SA * SA;
    kin[((size_t)mt * G + pp) * KST + e] = t.Kinv[((size_t)mt * g.P + q0 + pp) * SA * SA + e];
  }
  // per-thread angular tables
  T Ax[A][A], Ay[A][A];
  if (mine) {
#pragma unroll
    for (int m = 0; m < A; ++m)
#pragma unroll
      for (int dd = 0; dd < A; ++dd) {
        Ax[m][dd] = t.Aax[((size_t)q * 3 + 0) * A * A + m * A + dd];
        Ay[m][dd] = t.Aax[((size_t)q * 3 + 1) * A * A + m * A + dd];
      }
  }
  const int nchunk_seg = seg * (int)sizeof(T) / chunk;
  const int per_level = ny * S * nchunk_seg;
  // This thread's staging copies are the same (row, node, chunk) triples at
  // every level; only the cell column jx = w - row moves, so the source
  // address is linear in w.
  // UMAX: copy slots per thread and level, ceil(per_level / blockDim), <= 12
  int crow[UMAX];
  long long csrc[UMAX];
  int cdst[UMAX];
  int nu = 0;
  const long long xstep = (negx ? -1LL : 1LL) * S * nadof * (long long)sizeof(T);
#pragma unroll
  for (int u = 0; u < UMAX; ++u) {
    const int i = tid + u * (int)blockDim.x;
    crow[u] = -1;
    if (i < per_level) {
      const int row = i / (S * nchunk_seg);
      const int rem = i - row * S * nchunk_seg;
      const int l = rem / nchunk_seg, ch = rem - l * nchunk_seg;
      const int ix0 = negx ? nx - 1 : 0;  // column jx = 0
      const int iy = negy ? ny - 1 - row : row;
      const int c0 = ix0 + nx * iy;
      crow[u] = row;
      csrc[u] = (((long long)c0 * S + l) * nadof + q0 * A) * (long long)sizeof(T) + ch * chunk;
      cdst[u] = (int)(((size_t)row * S + l) * segp * sizeof(T)) + ch * chunk;
      nu = u + 1;
    }
  }
  const char* bbase = reinterpret_cast<const char*>(b);
  char* sbase = reinterpret_cast<char*>(stage);
  const int stage_bytes = ny * S * segp * (int)sizeof(T);
  auto issue = [&](int w) {
    if (w < sc.nlev) {
      char* st = sbase + (w % NST) * stage_bytes;
#pragma unroll
      for (int u = 0; u < UMAX; ++u) {
        if (u < nu) {
          const int jx = w - crow[u];
          if (jx >= 0 && jx < nx) cp_async_bytes(st + cdst[u], bbase + csrc[u] + jx * xstep, chunk);
        }
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int w = 0; w < NST - 1; ++w) issue(w);
  T xf[2][A];  // x-outflow of the previous cell of this row
  const int ownx = negx, owny = negy;
  const T fmx00 = T(g.facemass[0][0][0]), fmx01 = T(g.facemass[0][0][1]);
  const T fmx10 = T(g.facemass[0][1][0]), fmx11 = T(g.facemass[0][1][1]);
  const T fmy00 = T(g.facemass[1][0][0]), fmy01 = T(g.facemass[1][0][1]);
  const T fmy10 = T(g.facemass[1][1][0]), fmy11 = T(g.facemass[1][1][1]);
  const T nsx = ownx ? T(1) : T(-1), nsy = owny ? T(1) : T(-1);
  int mat_next = 0;
  if (mine) {
    const int ix = negx ? nx - 1 : 0, iy = negy ? ny - 1 - jy : jy;
    mat_next = cd.mat[ix + nx * iy];
  }
  for (int w = 0; w < sc.nlev; ++w) {
    cp_async_wait<NST - 2>();
    __syncthreads();
    issue(w + NST - 1);
    const int jx = w - jy;
    if (mine && jx >= 0 && jx < nx) {
      const int ix = negx ? nx - 1 - jx : jx;
      const int iy = negy ? ny - 1 - jy : jy;
      const int c = ix + nx * iy;
      const int mat = mat_next;
      if (jx + 1 < nx) mat_next = cd.mat[c + (negx ? -1 : 1)];
      T rhs[SA];
      const T* st = stage + (size_t)(w % NST) * ny * S * segp + (size_t)jy * S * segp + p * A;
#pragma unroll
      for (int l = 0; l < S; ++l)
#pragma unroll
        for (int m = 0; m < A; ++m) rhs[l * A + m] = st[l * segp + m];
      // Node l of the cell is on the x-inflow face when bit 0 of l equals
      // ownx (face index jp = bit 1 of l), on the y-inflow face when bit 1
      // equals owny (face index jp = bit 0).  Indices stay compile-time.
      if (jx > 0) {  // x-upwind from registers
        T dv[2][A];
#pragma unroll
        for (int jp = 0; jp < 2; ++jp)
#pragma unroll
          for (int m = 0; m < A; ++m) {
            T a0 = T(0), a1 = T(0);
#pragma unroll
            for (int dd = 0; dd < A; ++dd) {
              a0 += Ax[m][dd] * xf[0][dd];
              a1 += Ax[m][dd] * xf[1][dd];
            }
            dv[jp][m] = nsx * (jp == 0 ? fmx00 * a0 + fmx01 * a1 : fmx10 * a0 + fmx11 * a1);
          }
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const bool on = (l & 1) == ownx;
#pragma unroll
          for (int m = 0; m < A; ++m) rhs[l * A + m] -= on ? dv[l >> 1][m] : T(0);
        }
      }
      if (jy > 0) {  // y-upwind from row jy-1
        const T* yf = yface + ((size_t)((w - 1) & 1) * ny * G + (size_t)(jy - 1) * G + p) * 2 * A;
        T yv[2][A];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int m = 0; m < A; ++m) yv[j][m] = yf[j * A + m];
        T dv[2][A];
#pragma unroll
        for (int jp = 0; jp < 2; ++jp)
#pragma unroll
          for (int m = 0; m < A; ++m) {
            T a0 = T(0), a1 = T(0);
#pragma unroll
            for (int dd = 0; dd < A; ++dd) {
              a0 += Ay[m][dd] * yv[0][dd];
              a1 += Ay[m][dd] * yv[1][dd];
            }
            dv[jp][m] = nsy * (jp == 0 ? fmy00 * a0 + fmy01 * a1 : fmy10 * a0 + fmy11 * a1);
          }
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const bool on = ((l >> 1) & 1) == owny;
#pragma unroll
          for (int m = 0; m < A; ++m) rhs[l * A + m] -= on ? dv[l & 1][m] : T(0);
        }
      }
      // x = Kinv rhs (rows of SA values are 16-byte aligned in shared memory)
      T x[SA];
      if (mat < nmat_s) {
        const T* Ki = kin + ((size_t)mat * G + p) * KST;
#pragma unroll
        for (int r = 0; r < SA; ++r) {
          T acc = T(0);
#pragma unroll
          for (int cc = 0; cc < SA; cc += 16 / (int)sizeof(T)) {
            if constexpr (sizeof(T) == 4) {
              const float4 k4 = *reinterpret_cast<const float4*>(Ki + r * SA + cc);
              acc += k4.x * rhs[cc] + k4.y * rhs[cc + 1] + k4.z * rhs[cc + 2] + k4.w * rhs[cc + 3];
            } else {
              const double2 k2 = *reinterpret_cast<const double2*>(Ki + r * SA + cc);
              acc += k2.x * rhs[cc] + k2.y * rhs[cc + 1];
            }
          }
          x[r] = acc;
        }
      } else {
        const T* Ki = t.Kinv + ((size_t)mat * g.P + q) * SA * SA;
#pragma unroll
        for (int r = 0; r < SA; ++r) {
          T acc = T(0);
#pragma unroll
          for (int cc = 0; cc < SA; ++cc) acc += __ldg(Ki + r * SA + cc) * rhs[cc];
          x[r] = acc;
        }
      }
      T* out = psi + (long long)c * S * nadof + q * A;
#pragma unroll
      for (int l = 0; l < S; ++l)
#pragma unroll
        for (int m = 0; m < A; ++m) out[(long long)l * nadof + m] = x[l * A + m];
      // outflow faces for the next cell of this row and for row jy+1: nodes
      // with bit 0 (x) or bit 1 (y) equal to 1 - own
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int m = 0; m < A; ++m)
          xf[j][m] = ownx ? x[(2 * j) * A + m] : x[(2 * j + 1) * A + m];
      T* yo = yface + ((size_t)(w & 1) * ny * G + (size_t)jy * G + p) * 2 * A;
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int m = 0; m < A; ++m) yo[j * A + m] = owny ? x[j * A + m] : x[(2 + j) * A + m];
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// 2D sweep, warp-pipelined.  The task split is that of sweep2d_rows_kernel
// (one block per direction and patch group), without a block barrier per
// wavefront level: warp w owns the RW = 32 / G rows RW w .. RW w + RW - 1
// (lane = r G + p: row r, patch p) and runs its own steps t = 0, 1, ...,
// in which lane (r, p) solves cell jx = t - r of its row.  Row r > 0 takes its
// y-upwind values from row r - 1's output of the step before (a shuffle); row
// 0 takes them from the previous warp's last row through a ring of R cell
// slots in shared memory, published by a per-warp step counter (release /
// acquire at block scope); a writer reuses a slot only after the reader has
// passed it.  Every warp waits only on its two neighbours, and a writer at
// step t' needs its reader at step >= t' - RW + 2 - R while the reader at step
// t needs the writer at step >= t + RW, so no two warps wait on each other
// (R >= 2).  Waits give up after 2 s (status code 7, AMGT_ERR_DEVICE_TIMEOUT
// at the next amgt_sync) or as soon as another wait gave up.  b is staged per
// warp NST steps ahead with cp.async; the block inverses sit in shared memory.
__device__ __forceinline__ int ld_acquire_cta(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared.b32 %0, [%1];"
               : "=r"(v)
               : "r"((unsigned)__cvta_generic_to_shared(p))
               : "memory");
  return v;
}
__device__ __forceinline__ void st_release_cta(int* p, int v) {
  asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)),
               "r"(v)
               : "memory");
}
constexpr unsigned long long kSweepWaitNs = 2000000000ULL;
constexpr unsigned long long kSweepTestWaitNs = 10000000ULL;  // failure-path tests
// lane 0 waits until *p >= target; false once it gave up (after wait_ns, or
// as soon as another wait gave up)
__device__ __forceinline__ bool wait_at_least(const int* p, int target, int* err,
                                              unsigned long long wait_ns) {
  if (ld_acquire_cta(p) >= target) return true;
  const unsigned long long t0 = gsx::now_ns();
  unsigned it = 0;
  while (ld_acquire_cta(p) < target) {
    // after a few polls, back off: a spinning warp takes issue slots from the
    // warps it waits for
    if (it >= 4) __nanosleep(32);
    if ((++it & 63u) == 0) {
      if (*reinterpret_cast<volatile int*>(err) != 0) return false;
      if (gsx::now_ns() - t0 > wait_ns) {
        atomicExch(err, 7);
        return false;
      }
    }
  }
  return true;
}

constexpr int kSweepRing = 16;

// Row stride (elements) of a warp's staged rows [RW][S][G A]: the smallest
// 16-byte multiple >= S G A for which the reads of one (node, unknown) by the
// warp's lanes (row r, patch p: element r RS + p A) fall on distinct banks.
template <class T, int G, int A>
__host__ __device__ constexpr int warp_row_stride() {
  constexpr int S = 4, RW = 32 / G, vw = 16 / (int)sizeof(T), wpe = (int)sizeof(T) / 4;
  int best = S * G * A, bestc = 1 << 30;
  for (int k = 0; k < 8; ++k) {
    const int rs = ((S * G * A + vw - 1) / vw + k) * vw;
    int cnt[32] = {};
    int worst = 0;
    for (int r = 0; r < RW; ++r)
      for (int p = 0; p < G; ++p) {
        const int bank = ((r * rs + p * A) * wpe) % 32;
        const int c = ++cnt[bank];
        worst = c > worst ? c : worst;
      }
    if (worst < bestc) {
      bestc = worst;
      best = rs;
    }
  }
  return best;
}

template <class T>
size_t sweep2d_warp_smem(int ny, int G, int a, int nmat_s, int nst) {
  const int RW = 32 / G, nwarp = (ny + RW - 1) / RW;
  const int SA = 4 * a;
  const size_t kst = SA * SA + 16 / sizeof(T);
  const int rs = G == 2 ? warp_row_stride<T, 2, 3>()
                        : (G == 4 ? warp_row_stride<T, 4, 3>() : warp_row_stride<T, 8, 3>());
  return ((size_t)nwarp * (nst + 1) * RW * rs + (size_t)nwarp * kSweepRing * G * 2 * a +
          (size_t)nmat_s * G * kst) * sizeof(T) + (size_t)nwarp * sizeof(int);
}

template <class T, int A, int G, int NST, int UMAX>
__global__ void __launch_bounds__(512) sweep2d_warp_kernel(Geom g, LevelDev<T> t, CellData cd,
                                                            Schedule sc, const T* __restrict__ b,
                                                            T* __restrict__ psi, int nmat_s,
                                                            int chunk, int* err,
                                                            unsigned long long wait_ns,
                                                            int hold) {
  constexpr int S = 4, HS = 2;
  constexpr int SA = S * A;
  constexpr int RW = 32 / G;
  constexpr int SEGP = G * A;                    // (row, node) segment
  constexpr int RS = warp_row_stride<T, G, A>();  // staged row stride
  constexpr int KST = SA * SA + 16 / sizeof(T);  // padded inverse stride
  constexpr int R = kSweepRing;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int task = blockIdx.x;
  const int d = sc.task_dir[task], q0 = sc.task_q0[task], nq = sc.task_nq[task];
  const int negx = (d >> 1) & 1, negy = d & 1;
  const int nx = g.nx, ny = g.ny, nadof = g.nadof;
  const int nwarp = blockDim.x >> 5;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = lane / G, p = lane - (lane / G) * G;
  const int jy = warp * RW + r;
  const bool mine = jy < ny && p < nq;
  const int q = q0 + p;
  const int seg = nq * A;
  T* stage = reinterpret_cast<T*>(smem_raw);                 // [nwarp][NST + 1][RW][RS]
  T* ring = stage + (size_t)nwarp * (NST + 1) * RW * RS;    // [nwarp][R][G][HS*A]
  T* kin = ring + (size_t)nwarp * R * G * HS * A;                  // [nmat_s][G][KST]
  int* prog = reinterpret_cast<int*>(kin + (size_t)nmat_s * G * KST);  // [nwarp] steps done
  for (int i = tid; i < nmat_s * nq * SA * SA; i += blockDim.x) {
    const int mt = i / (nq * SA * SA);
    const int rem = i - mt * nq * SA * SA;
    const int pp = rem / (SA * SA), e = rem - pp * SA * SA;
    kin[((size_t)mt * G + pp) * KST + e] = t.Kinv[((size_t)mt * g.P + q0 + pp) * SA * SA + e];
  }
  if (tid < nwarp) prog[tid] = 0;
  T Ax[A][A], Ay[A][A];
  if (mine) {
#pragma unroll
    for (int m = 0; m < A; ++m)
#pragma unroll
      for (int dd = 0; dd < A; ++dd) {
        Ax[m][dd] = t.Aax[((size_t)q * 3 + 0) * A * A + m * A + dd];
        Ay[m][dd] = t.Aax[((size_t)q * 3 + 1) * A * A + m * A + dd];
      }
  }
  // this lane's staging copies: the same (row, node, chunk) triples every
  // step; the cell column jx = step - row moves, linear in the source address
  const int nchunk_seg = seg * (int)sizeof(T) / chunk;
  const int per_step = RW * S * nchunk_seg;
  int crow[UMAX];
  long long csrc[UMAX];
  int cdst[UMAX];
  const long long xstep = (negx ? -1LL : 1LL) * S * nadof * (long long)sizeof(T);
#pragma unroll
  for (int u = 0; u < UMAX; ++u) {
    const int i = lane + u * 32;
    crow[u] = -1;
    csrc[u] = 0;
    cdst[u] = 0;
    if (i < per_step) {
      const int row = i / (S * nchunk_seg);
      const int rem = i - row * S * nchunk_seg;
      const int l = rem / nchunk_seg, ch = rem - l * nchunk_seg;
      const int jyc = warp * RW + row;
      if (jyc < ny) {
        const int iy = negy ? ny - 1 - jyc : jyc;
        const int c0 = (negx ? nx - 1 : 0) + nx * iy;
        crow[u] = row;
        csrc[u] = (((long long)c0 * S + l) * nadof + q0 * A) * (long long)sizeof(T) + ch * chunk;
        cdst[u] = (row * RS + l * SEGP) * (int)sizeof(T) + ch * chunk;
      }
    }
  }
  const char* bbase = reinterpret_cast<const char*>(b);
  constexpr int kStageElems = RW * RS;
  T* wstage = stage + (size_t)warp * (NST + 1) * kStageElems;
  T* wout = wstage + (size_t)NST * kStageElems;  // this warp's outputs of one step
  char* wbase = reinterpret_cast<char*>(wstage);
  // outputs leave through the staging buffer as whole 16- or 8-byte chunks
  // when the segments are so aligned (the copy layout of b)
  const bool vec_out = chunk >= 8;
  const int nsteps = nx + RW - 1;
  auto issue = [&](int ts) {
    if (ts < nsteps) {
      char* st = wbase + (ts % NST) * kStageElems * (int)sizeof(T);
#pragma unroll
      for (int u = 0; u < UMAX; ++u) {
        if (crow[u] >= 0) {
          const int jx = ts - crow[u];
          if (jx >= 0 && jx < nx) cp_async_bytes(st + cdst[u], bbase + csrc[u] + jx * xstep, chunk);
        }
      }
    }
    cp_async_commit();
  };
  __syncthreads();
#pragma unroll
  for (int ts = 0; ts < NST - 1; ++ts) issue(ts);
  const int ownx = negx, owny = negy;
  const T fmx00 = T(g.facemass[0][0][0]), fmx01 = T(g.facemass[0][0][1]);
  const T fmx10 = T(g.facemass[0][1][0]), fmx11 = T(g.facemass[0][1][1]);
  const T fmy00 = T(g.facemass[1][0][0]), fmy01 = T(g.facemass[1][0][1]);
  const T fmy10 = T(g.facemass[1][1][0]), fmy11 = T(g.facemass[1][1][1]);
  const T nsx = ownx ? T(1) : T(-1), nsy = owny ? T(1) : T(-1);
  T xf[HS][A], yo[HS][A];
#pragma unroll
  for (int j = 0; j < HS; ++j)
#pragma unroll
    for (int m = 0; m < A; ++m) {
      xf[j][m] = T(0);
      yo[j][m] = T(0);
    }
  const int iy = negy ? ny - 1 - jy : jy;
  int mat_next = 0;
  if (mine) mat_next = cd.mat[(negx ? nx - 1 : 0) + nx * iy];
  for (int ts = 0; ts < nsteps; ++ts) {
    cp_async_wait<NST - 2>();
    __syncwarp();
    issue(ts + NST - 1);
    const int jx = ts - r;
    const bool act = mine && jx >= 0 && jx < nx;
    // y-upwind values: row r - 1's outputs of the step before
    T yv[HS][A];
#pragma unroll
    for (int j = 0; j < HS; ++j)
#pragma unroll
      for (int m = 0; m < A; ++m) yv[j][m] = __shfl_up_sync(0xffffffffu, yo[j][m], G);
    // row 0: the previous warp's last row, once that warp has passed step ts + RW - 1
    if (warp > 0 && ts < nx) {
      bool ok = true;
      if (lane == 0) ok = wait_at_least(prog + warp - 1, ts + RW, err, wait_ns);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      __syncwarp();  // lane 0's acquire orders the ring reads of every lane
      if (r == 0 && p < nq) {
        const T* rs = ring + (((size_t)(warp - 1) * R + ts % R) * G + p) * HS * A;
#pragma unroll
        for (int j = 0; j < HS; ++j)
#pragma unroll
          for (int m = 0; m < A; ++m) yv[j][m] = rs[j * A + m];
      }
    }
    if (act) {
      const int ix = negx ? nx - 1 - jx : jx;
      const int c = ix + nx * iy;
      const int mat = mat_next;
      if (jx + 1 < nx) mat_next = cd.mat[c + (negx ? -1 : 1)];
      T rhs[SA];
      const T* st = wstage + (size_t)(ts % NST) * kStageElems + (size_t)r * RS + p * A;
#pragma unroll
      for (int l = 0; l < S; ++l)
#pragma unroll
        for (int m = 0; m < A; ++m) rhs[l * A + m] = st[l * SEGP + m];
      // node l is on the x-inflow face when bit 0 of l equals ownx (face index
      // bit 1 of l), on the y-inflow face when bit 1 equals owny (bit 0)
      if (jx > 0) {
        T dv[HS][A];
#pragma unroll
        for (int jp = 0; jp < HS; ++jp)
#pragma unroll
          for (int m = 0; m < A; ++m) {
            T a0 = T(0), a1 = T(0);
#pragma unroll
            for (int dd = 0; dd < A; ++dd) {
              a0 += Ax[m][dd] * xf[0][dd];
              a1 += Ax[m][dd] * xf[1][dd];
            }
            dv[jp][m] = nsx * (jp == 0 ? fmx00 * a0 + fmx01 * a1 : fmx10 * a0 + fmx11 * a1);
          }
#pragma unroll
        for (int l = 0; l < S; ++l) {
          const bool on = (l & 1) == ownx;
#pragma unroll
          for (int m = 0; m < A; ++m) rhs[l * A + m] -= on ? dv[l >> 1][m] : T(0);
        }
      }
      if (jy > 0) {
        T dv[HS][A];
#pragma unroll
        for (int jp = 0; jp < HS; ++jp)
#pragma unroll
          for (int m = 0; m < A; ++m) {
            T a0 = T(0), a1 = T(0);
#pragma unroll
            for (int dd = 0; dd < A; ++dd) {
              a0 += Ay[m][dd] * yv[0][dd];
              a1 += Ay[m][dd] * yv[1][dd];
            }
            dv[jp][m] = nsy * (jp == 0 ? fmy00 * a0 + fmy01 * a1 : fmy10 * a0 + fmy11 * a1);
          }
#pragma unroll
        for (int l = 0; l < S; ++l) {
          const bool on = ((l >> 1) & 1) == owny;
#pragma unroll
          for (int m = 0; m < A; ++m) rhs[l * A + m] -= on ? dv[l & 1][m] : T(0);
        }
      }
      T x[SA];
      if (mat < nmat_s) {
        const T* Ki = kin + ((size_t)mat * G + p) * KST;
#pragma unroll
        for (int rr = 0; rr < SA; ++rr) {
          T acc = T(0);
#pragma unroll
          for (int cc = 0; cc < SA; cc += 16 / (int)sizeof(T)) {
            if constexpr (sizeof(T) == 4) {
              const float4 k4 = *reinterpret_cast<const float4*>(Ki + rr * SA + cc);
              acc += k4.x * rhs[cc] + k4.y * rhs[cc + 1] + k4.z * rhs[cc + 2] + k4.w * rhs[cc + 3];
            } else {
              const double2 k2 = *reinterpret_cast<const double2*>(Ki + rr * SA + cc);
              acc += k2.x * rhs[cc] + k2.y * rhs[cc + 1];
            }
          }
          x[rr] = acc;
        }
      } else {
        const T* Ki = t.Kinv + ((size_t)mat * g.P + q) * SA * SA;
#pragma unroll
        for (int rr = 0; rr < SA; ++rr) {
          T acc = T(0);
#pragma unroll
          for (int cc = 0; cc < SA; ++cc) acc += __ldg(Ki + rr * SA + cc) * rhs[cc];
          x[rr] = acc;
        }
      }
      if (vec_out) {
        T* o = wout + (size_t)r * RS + p * A;
#pragma unroll
        for (int l = 0; l < S; ++l)
#pragma unroll
          for (int m = 0; m < A; ++m) o[l * SEGP + m] = x[l * A + m];
      } else {
        T* out = psi + (long long)c * S * nadof + q * A;
#pragma unroll
        for (int l = 0; l < S; ++l)
#pragma unroll
          for (int m = 0; m < A; ++m) out[(long long)l * nadof + m] = x[l * A + m];
      }
      // outflow faces: nodes with bit 0 (x) or bit 1 (y) equal to 1 - own
#pragma unroll
      for (int j = 0; j < HS; ++j)
#pragma unroll
        for (int m = 0; m < A; ++m) {
          xf[j][m] = ownx ? x[(2 * j) * A + m] : x[(2 * j + 1) * A + m];
          yo[j][m] = owny ? x[j * A + m] : x[(2 + j) * A + m];
        }
    }
    if (vec_out) {
      // the step's outputs as 16-byte chunks: the same (row, node, chunk)
      // triples as the copies of b, each to its cell's segment of psi
      __syncwarp();
      char* pbase = reinterpret_cast<char*>(psi);
      const char* obase = reinterpret_cast<const char*>(wout);
#pragma unroll
      for (int u = 0; u < UMAX; ++u) {
        if (crow[u] >= 0) {
          const int jx2 = ts - crow[u];
          if (jx2 >= 0 && jx2 < nx) {
            if (chunk == 16)
              *reinterpret_cast<int4*>(pbase + csrc[u] + jx2 * xstep) =
                  *reinterpret_cast<const int4*>(obase + cdst[u]);
            else
              *reinterpret_cast<int2*>(pbase + csrc[u] + jx2 * xstep) =
                  *reinterpret_cast<const int2*>(obase + cdst[u]);
          }
        }
      }
    }
    // the last row's outputs into the ring for the next warp
    const int jl = ts - (RW - 1);
    if (warp + 1 < nwarp && jl >= 0 && jl < nx) {
      bool ok = true;
      if (lane == 0 && jl >= R) ok = wait_at_least(prog + warp + 1, jl - R + 1, err, wait_ns);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      if (r == RW - 1 && p < nq && jy < ny) {
        T* rs = ring + (((size_t)warp * R + jl % R) * G + p) * HS * A;
#pragma unroll
        for (int j = 0; j < HS; ++j)
#pragma unroll
          for (int m = 0; m < A; ++m) rs[j * A + m] = yo[j][m];
      }
    }
    __syncwarp();
    // (hold: the failure-path test keeps warp 0's progress unpublished)
    if (lane == 0 && !(hold && warp == 0)) st_release_cta(prog + warp, ts + 1);
  }
  cp_async_wait<0>();
}

// Spatial matrices of the Kronecker form of the diagonal block
//   K0_q + sigma_t kron(N, M_q) = sum_xi kron(G_xi^(sign), A^xi_q) + sigma_t kron(N, M_q),
//   G_xi^(+) = Fown_{xi,high} - V_xi,   G_xi^(-) = -Fown_{xi,low} - V_xi,
// where the sign is that of Omega_xi on the patch (one outflow face per axis).
template <class T>
__device__ __forceinline__ T gax(const Geom& g, int xi, int sg, int e);
template <>
__device__ __forceinline__ double gax<double>(const Geom& g, int xi, int sg, int e) {
  return g.Gax[xi][sg][e];
}
template <>
__device__ __forceinline__ float gax<float>(const Geom& g, int xi, int sg, int e) {
  return g.GaxF[xi][sg][e];
}
template <class T>
__device__ __forceinline__ T nsp(const Geom& g, int e);
template <>
__device__ __forceinline__ double nsp<double>(const Geom& g, int e) { return g.Nmass[e]; }
template <>
__device__ __forceinline__ float nsp<float>(const Geom& g, int e) { return g.NmassF[e]; }

// three blocks per SM for the 2D FP32 form; two (up to 128 registers, no
// spills of the wider FP64 working set) otherwise
template <class T, int DIM, int A>
__global__ void __launch_bounds__(256, DIM == 2 && sizeof(T) == 4 ? 3 : 2) apply_L_kernel(Geom g, LevelDev<T> t, CellData cd,
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
    T xv[S][A];
#pragma unroll
    for (int l = 0; l < S; ++l)
#pragma unroll
      for (int m = 0; m < A; ++m) xv[l][m] = xp[(long long)l * nadof + m];
    T acc[SA];
#pragma unroll
    for (int r = 0; r < SA; ++r) acc[r] = T(0);
    // streaming: sum_xi G_xi X (A^xi)^T
#pragma unroll
    for (int xi = 0; xi < DIM; ++xi) {
      const T* Aq = t.Aax + ((size_t)q * 3 + xi) * A * A;
      T a[A][A];
#pragma unroll
      for (int m = 0; m < A; ++m)
#pragma unroll
        for (int d = 0; d < A; ++d) a[m][d] = Aq[m * A + d];
      T t1[S][A];
#pragma unroll
      for (int i = 0; i < S; ++i)
#pragma unroll
        for (int m = 0; m < A; ++m) {
          T v = T(0);
#pragma unroll
          for (int d = 0; d < A; ++d) v += xv[i][d] * a[m][d];
          t1[i][m] = v;
        }
      const int sg = neg[xi];
#pragma unroll
      for (int l = 0; l < S; ++l)
#pragma unroll
        for (int i = 0; i < S; ++i) {
          const T gli = gax<T>(g, xi, sg, l * S + i);
#pragma unroll
          for (int m = 0; m < A; ++m) acc[l * A + m] += gli * t1[i][m];
        }
    }
    // collision: sigma_t N X M^T
    {
      const T st = (T)cd.sigma_t[c];
      const T* Mm = t.Mang + (size_t)q * A * A;
      T t1[S][A];
#pragma unroll
      for (int i = 0; i < S; ++i)
#pragma unroll
        for (int m = 0; m < A; ++m) {
          T v = T(0);
#pragma unroll
          for (int d = 0; d < A; ++d) v += xv[i][d] * Mm[m * A + d];
          t1[i][m] = st * v;
        }
#pragma unroll
      for (int l = 0; l < S; ++l)
#pragma unroll
        for (int i = 0; i < S; ++i) {
          const T nli = nsp<T>(g, l * S + i);
#pragma unroll
          for (int m = 0; m < A; ++m) acc[l * A + m] += nli * t1[i][m];
        }
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

// y = alpha L x + beta y to FP64 accuracy on the FP32 units: the Kronecker
// form of apply_L_kernel in double-float arithmetic.  x, y and sigma_t are
// split by integer operations, the patch tables A^xi_q and M_q come split
// (hi, lo) from set-up, and the geometric constants are split once per block
// into shared memory, so the only FP64 instruction is the final hi + lo of
// each output.  In 2D two blocks per SM (128 registers, a few spilled)
// measured 13% faster than one block without spills.
template <int DIM, int A>
__global__ void __launch_bounds__(256, DIM == 2 ? 2 : 1)
    apply_L_df_kernel(Geom g, const float2* __restrict__ aax, const float2* __restrict__ mang,
                      const int* __restrict__ pdir, const double* __restrict__ sigma_t,
                      double alpha, double beta, const double* __restrict__ x,
                      double* __restrict__ y) {
  constexpr int S = 1 << DIM, HS = S / 2, SA = S * A;
  __shared__ float2 sG[DIM][2][S * S];  // streaming matrices G_xi^(sign)
  __shared__ float2 sN[S * S];          // spatial mass N
  __shared__ float2 sF[DIM][HS][HS];    // face masses
  for (int i = threadIdx.x; i < DIM * 2 * S * S + S * S + DIM * HS * HS; i += blockDim.x) {
    double v;
    float2* dst;
    if (i < DIM * 2 * S * S) {
      const int xi = i / (2 * S * S), sg = (i / (S * S)) & 1, e = i % (S * S);
      v = g.Gax[xi][sg][e];
      dst = &sG[xi][sg][e];
    } else if (i < DIM * 2 * S * S + S * S) {
      const int e = i - DIM * 2 * S * S;
      v = g.Nmass[e];
      dst = &sN[e];
    } else {
      const int e = i - DIM * 2 * S * S - S * S;
      const int xi = e / (HS * HS), jp = (e / HS) % HS, j = e % HS;
      v = g.facemass[xi][jp][j];
      dst = &sF[xi][jp][j];
    }
    const float h = (float)v;
    *dst = make_float2(h, (float)(v - (double)h));
  }
  __syncthreads();
  const DF alpha_df(alpha), beta_df(beta);
  const bool unit_alpha = alpha == 1.0;
  const long long total = (long long)g.C * g.P;
  const int nadof = g.nadof;
  const int stride[3] = {1, g.nx, g.nx * g.ny};
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / g.P);
    const int q = (int)(idx - (long long)c * g.P);
    int neg[3];
    dir_bits<DIM>(pdir[q], neg);
    const int ix = c % g.nx, iy = (c / g.nx) % g.ny, iz = c / (g.nx * g.ny);
    const int jj[3] = {neg[0] ? g.nx - 1 - ix : ix, neg[1] ? g.ny - 1 - iy : iy,
                       neg[2] ? g.nz - 1 - iz : iz};
    const double* xp = x + (long long)c * S * nadof + q * A;
    DF xv[S][A];
#pragma unroll
    for (int l = 0; l < S; ++l)
#pragma unroll
      for (int m = 0; m < A; ++m) xv[l][m] = df_split(xp[(long long)l * nadof + m]);
    DFAcc acc[SA];
    // streaming: sum_xi G_xi X (A^xi)^T
#pragma unroll
    for (int xi = 0; xi < DIM; ++xi) {
      const float2* Aq = aax + ((size_t)q * 3 + xi) * A * A;
      DF a[A][A];
#pragma unroll
      for (int m = 0; m < A; ++m)
#pragma unroll
        for (int d = 0; d < A; ++d) {
          const float2 v = Aq[m * A + d];
          a[m][d] = DF(v.x, v.y);
        }
      const int sg = neg[xi];
#pragma unroll
      for (int i = 0; i < S; ++i) {
        DF t1[A];
#pragma unroll
        for (int m = 0; m < A; ++m) {
          DFAcc v;
#pragma unroll
          for (int d = 0; d < A; ++d) df_fma(v, xv[i][d], a[m][d]);
          t1[m] = df_val(v);
        }
#pragma unroll
        for (int l = 0; l < S; ++l) {
          const float2 gv = sG[xi][sg][l * S + i];
          const DF gli(gv.x, gv.y);
#pragma unroll
          for (int m = 0; m < A; ++m) df_fma(acc[l * A + m], gli, t1[m]);
        }
      }
    }
    // collision: sigma_t N X M^T
    {
      const DF st = df_split(sigma_t[c]);
      const float2* Mm = mang + (size_t)q * A * A;
      DF mq[A][A];
#pragma unroll
      for (int m = 0; m < A; ++m)
#pragma unroll
        for (int d = 0; d < A; ++d) {
          const float2 v = Mm[m * A + d];
          mq[m][d] = DF(v.x, v.y);
        }
#pragma unroll
      for (int i = 0; i < S; ++i) {
        DF t1[A];
#pragma unroll
        for (int m = 0; m < A; ++m) {
          DFAcc v;
#pragma unroll
          for (int d = 0; d < A; ++d) df_fma(v, xv[i][d], mq[m][d]);
          t1[m] = st * df_val(v);
        }
#pragma unroll
        for (int l = 0; l < S; ++l) {
          const float2 nv = sN[l * S + i];
          const DF nli(nv.x, nv.y);
#pragma unroll
          for (int m = 0; m < A; ++m) df_fma(acc[l * A + m], nli, t1[m]);
        }
      }
    }
    // inflow faces: sum over f of kron(Fnb_f, A_{f,q}) x_nb, A_{f,q} = n_xi A^xi_q
#pragma unroll
    for (int xi = 0; xi < DIM; ++xi) {
      if (jj[xi] == 0) continue;
      const int own = neg[xi];
      const int cn = c + (own ? stride[xi] : -stride[xi]);
      const float2* An = aax + ((size_t)q * 3 + xi) * A * A;
      const double* pn = x + (long long)cn * S * nadof + q * A;
      DF tv[HS][A];
#pragma unroll
      for (int j = 0; j < HS; ++j) {
        const int i = fnode(j, xi, 1 - own);
        DF v[A];
#pragma unroll
        for (int d = 0; d < A; ++d) v[d] = df_split(pn[(long long)i * nadof + d]);
#pragma unroll
        for (int m = 0; m < A; ++m) {
          DFAcc sacc;
#pragma unroll
          for (int d = 0; d < A; ++d) {
            const float2 av = An[m * A + d];
            df_fma(sacc, DF(av.x, av.y), v[d]);
          }
          const DF t = df_val(sacc);
          tv[j][m] = own ? t : -t;  // outward normal component
        }
      }
#pragma unroll
      for (int jp = 0; jp < HS; ++jp) {
        const int l = fnode(jp, xi, own);
#pragma unroll
        for (int j = 0; j < HS; ++j) {
          const float2 fv = sF[xi][jp][j];
          const DF fm(fv.x, fv.y);
#pragma unroll
          for (int m = 0; m < A; ++m) df_fma(acc[l * A + m], fm, tv[j][m]);
        }
      }
    }
    double* out = y + (long long)c * S * nadof + q * A;
#pragma unroll
    for (int r = 0; r < SA; ++r) {
      double* o = out + (long long)(r / A) * nadof + (r % A);
      DF v = df_val(acc[r]);
      if (!unit_alpha) v = alpha_df * v;
      if (beta != 0.0) v += beta_df * df_split(*o);
      *o = df_to_double(v);
    }
  }
}

// f[c*s+l][q*a+m] = q_c/(4 pi) mu_l w_qm + boundary inflow terms (isotropic
// inflow from the per-patch current integrals Aw, the pencil beam from its
// per-face table)
template <class T>
__global__ void source_kernel(Geom g, const T* __restrict__ w, const T* __restrict__ Aw,
                              const int* __restrict__ octant, const double* __restrict__ qsrc,
                              const double* __restrict__ bval, const int* __restrict__ bkind,
                              const double* __restrict__ beam,
                              const double* __restrict__ brange,
                              const double* __restrict__ mu, const double* __restrict__ mf,
                              T* __restrict__ f) {
  // one thread per (cell, patch): the cell's position, emission and boundary
  // faces once, then its s x a entries
  const long long total = (long long)g.C * g.P;
  const int a = g.a, s = g.s;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / g.P);
    const int q = (int)(idx - (long long)c * g.P);
    const double qc = qsrc[c] / (4.0 * M_PI);
    const int ic[3] = {c % g.nx, (c / g.nx) % g.ny, c / (g.nx * g.ny)};
    const int n[3] = {g.nx, g.ny, g.nz};
    const int o = octant[q];
    const int negb[3] = {(o >> 2) & 1, (o >> 1) & 1, o & 1};
    for (int l = 0; l < s; ++l) {
      for (int m = 0; m < a; ++m) {
        const int j = q * a + m;
        double v = qc * mu[l] * (double)w[j];
        for (int xi = 0; xi < g.dim; ++xi) {
          for (int side = 0; side < 2; ++side) {
            const int face = 2 * xi + side;
            if (bkind[face] == 0) continue;
            if (side == 0 ? ic[xi] != 0 : ic[xi] != n[xi] - 1) continue;
            if (bkind[face] == 2) {  // pencil beam: S mf_l Psi_m(Omega_b) share_q
              v += beam[(size_t)face * g.nadof + j] * mf[face * s + l];
              continue;
            }
            if (bkind[face] == 3) {
              // beam over part of the face: S |Omega_b.n| Psi_m(Omega_b) share_q times
              // the integral of Phi_l over the cell face and the range, a product
              // over the tangential axes of integrals of the linear nodal functions
              // l_0 = 1 - t/h, l_1 = t/h over the overlap [ta, tb] of the cell
              if (((l >> xi) & 1) != side) continue;
              double I = 1.0;
              int k = 0;
              for (int e = 0; e < g.dim; ++e) {
                if (e == xi) continue;
                const double x0 = g.lo[e] + ic[e] * g.h[e];
                const double lo_ = fmax(x0, brange[face * 4 + 2 * k]);
                const double hi_ = fmin(x0 + g.h[e], brange[face * 4 + 2 * k + 1]);
                ++k;
                if (!(hi_ > lo_)) {
                  I = 0.0;
                  break;
                }
                const double ta = lo_ - x0, tb = hi_ - x0, he = g.h[e];
                const double i1 = (tb * tb - ta * ta) / (2.0 * he);
                I *= ((l >> e) & 1) ? i1 : (tb - ta) - i1;
              }
              v += beam[(size_t)face * g.nadof + j] * I;
              continue;
            }
            // inflow iff the patch moves into the domain through this face
            const bool inflow = side == 0 ? (negb[xi] == 0) : (negb[xi] == 1);
            if (!inflow) continue;
            const double nsgn = side ? 1.0 : -1.0;
            v += -bval[face] * mf[face * s + l] * nsgn * (double)Aw[((size_t)q * 3 + xi) * a + m];
          }
        }
        f[((long long)c * s + l) * g.nadof + j] = (T)v;
      }
    }
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

// Uniform refinement with Lin patches (coarse patch c has the children
// 4c..4c+3, 3 functions each): a thread per coarse patch over a band of
// rows, its children's 4 x 3 x 3 coefficients in registers for the whole
// band, the 12 fine values of a row moved as 16-byte vectors (48 c bytes from
// a 16-byte aligned row start).
__device__ __forceinline__ void ld12(const float* p, float (&v)[12]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float4 q = reinterpret_cast<const float4*>(p)[i];
    v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
  }
}
__device__ __forceinline__ void ld12(const double* p, double (&v)[12]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const double2 q = reinterpret_cast<const double2*>(p)[i];
    v[2 * i] = q.x; v[2 * i + 1] = q.y;
  }
}
__device__ __forceinline__ void st12(float* p, const float (&v)[12]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
    reinterpret_cast<float4*>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
__device__ __forceinline__ void st12(double* p, const double (&v)[12]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) reinterpret_cast<double2*>(p)[i] = make_double2(v[2 * i], v[2 * i + 1]);
}

// rc[r][(c,d)] = sum over the children f = 4c + j and k of blk[f][k][d] rf[r][(f,k)]
template <class T>
__global__ void __launch_bounds__(256) restrict4_kernel(long long nsdof, int Pc, int rows_per_block,
                                                       const T* __restrict__ blk,
                                                       const T* __restrict__ rf,
                                                       T* __restrict__ rc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Pc) return;
  T b[36];
#pragma unroll
  for (int i = 0; i < 36; ++i) b[i] = blk[(size_t)c * 36 + i];
  const long long r0 = (long long)blockIdx.y * rows_per_block;
  const long long r1 = r0 + rows_per_block < nsdof ? r0 + rows_per_block : nsdof;
  const long long nf = 12LL * Pc, nc = 3LL * Pc;
#pragma unroll 4
  for (long long r = r0; r < r1; ++r) {
    T v[12];
    ld12(rf + r * nf + 12LL * c, v);
    T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int fk = 0; fk < 12; ++fk)
#pragma unroll
      for (int d = 0; d < 3; ++d) acc[d] += b[fk * 3 + d] * v[fk];
    T* o = rc + r * nc + 3LL * c;
    o[0] = acc[0];
    o[1] = acc[1];
    o[2] = acc[2];
  }
}

// xf[r][(f,k)] += sum_d blk[f][k][d] xc[r][(c,d)] for the children f = 4c + j
template <class T>
__global__ void __launch_bounds__(256) prolong4_kernel(long long nsdof, int Pc, int rows_per_block,
                                                      const T* __restrict__ blk,
                                                      const T* __restrict__ xc,
                                                      T* __restrict__ xf) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Pc) return;
  T b[36];
#pragma unroll
  for (int i = 0; i < 36; ++i) b[i] = blk[(size_t)c * 36 + i];
  const long long r0 = (long long)blockIdx.y * rows_per_block;
  const long long r1 = r0 + rows_per_block < nsdof ? r0 + rows_per_block : nsdof;
  const long long nf = 12LL * Pc, nc = 3LL * Pc;
#pragma unroll 2
  for (long long r = r0; r < r1; ++r) {
    const T* xr = xc + r * nc + 3LL * c;
    const T x0 = xr[0], x1 = xr[1], x2 = xr[2];
    T v[12];
    T* o = xf + r * nf + 12LL * c;
    ld12(o, v);
#pragma unroll
    for (int fk = 0; fk < 12; ++fk) v[fk] += b[fk * 3] * x0 + b[fk * 3 + 1] * x1 + b[fk * 3 + 2] * x2;
    st12(o, v);
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

}  // namespace


namespace {

int grid_for(long long total, int block) {
  long long g = (total + block - 1) / block;
  if (g > 152LL * 32) g = 152LL * 32;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

template <class T>
size_t sweep2d_smem(const Geom& g, int G, int nmat_s, int nst) {
  const int SA = 4 * g.a;
  const size_t kst = SA * SA + 16 / sizeof(T);
  return ((size_t)nst * g.ny * 4 * G * g.a + (size_t)2 * g.ny * G * 2 * g.a +
          (size_t)nmat_s * G * kst) * sizeof(T);
}

template <class T>
void launch_sweep(const Geom& g, const LevelDev<T>& t, const CellData& cd, const Schedule& sc,
                  const T* b, T* psi, int G, int nmat, int chunk_bytes, int nst, int variant,
                  int* err, int test_hold, unsigned* gbar, cudaStream_t st) {
  note_launch();
  // warp-pipelined form (variant 2; auto with at least 2 (FP32) or 4 (FP64)
  // patches per block, where it measured faster):
  // Lin basis, G dividing 32 with at least two patches per row, at most 512
  // threads
  const bool want_warp = variant == 2 || (variant == 0 && G >= (sizeof(T) == 4 ? 2 : 4));
  if (g.dim == 2 && want_warp && g.a == 3 && (G == 2 || G == 4 || G == 8) && err) {
    const int RW = 32 / G, nwarp = (g.ny + RW - 1) / RW;
    constexpr int NSTW = sizeof(T) == 4 ? 4 : 3;
    int nmat_s = nmat;
    while (nmat_s > 0 && sweep2d_warp_smem<T>(g.ny, G, 3, nmat_s, NSTW) > 200 * 1024) --nmat_s;
    const size_t smem = sweep2d_warp_smem<T>(g.ny, G, 3, nmat_s, NSTW);
    const int chunk = chunk_bytes > 0 ? chunk_bytes : (int)sizeof(T);
    const int seg_chunks = (G * 3 * (int)sizeof(T)) / chunk;
    const int need = (RW * 4 * seg_chunks + 31) / 32;
    if (nwarp * 32 <= 512 && smem <= 200 * 1024 && need <= 12) {
      auto launch = [&](auto kern) {
        allow_max_smem(kern);
        kern<<<sc.ntask, nwarp * 32, smem, st>>>(g, t, cd, sc, b, psi, nmat_s, chunk, err,
                                                 test_hold ? kSweepTestWaitNs : kSweepWaitNs,
                                                 test_hold ? 1 : 0);
      };
      auto by_g = [&](auto g_tag) {
        constexpr int GG = decltype(g_tag)::value;
        if (need <= 3) launch(sweep2d_warp_kernel<T, 3, GG, NSTW, 3>);
        else if (need <= 6) launch(sweep2d_warp_kernel<T, 3, GG, NSTW, 6>);
        else launch(sweep2d_warp_kernel<T, 3, GG, NSTW, 12>);
      };
      if (G == 2) by_g(std::integral_constant<int, 2>());
      else if (G == 4) by_g(std::integral_constant<int, 4>());
      else by_g(std::integral_constant<int, 8>());
      return;
    }
  }
  if (g.dim == 2 && G > 0 && g.ny * G <= 512) {
    int NST = nst > 0 ? nst : (sizeof(T) == 4 ? 4 : 3);
    NST = NST >= 6 ? 6 : (NST >= 4 ? 4 : (NST >= 3 ? 3 : 2));
    while (NST > 2 && sweep2d_smem<T>(g, G, 0, NST) > 200 * 1024) NST = NST == 6 ? 4 : NST - 1;
    int nmat_s = nmat;
    while (nmat_s > 0 && sweep2d_smem<T>(g, G, nmat_s, NST) > 200 * 1024) --nmat_s;
    const size_t smem = sweep2d_smem<T>(g, G, nmat_s, NST);
    // 16-byte copies when every segment start and length is 16-byte aligned
    const int chunk = chunk_bytes > 0 ? chunk_bytes : (int)sizeof(T);
    const int threads = ((g.ny * G + 31) / 32) * 32;
    const int seg_chunks = (G * g.a * (int)sizeof(T) + chunk - 1) / chunk;
    const bool slots_ok = (long long)g.ny * 4 * seg_chunks <= 12LL * threads;
    if (smem <= 200 * 1024 && slots_ok) {
      auto launch = [&](auto kern) {
        allow_max_smem(kern);
        kern<<<sc.ntask, threads, smem, st>>>(g, t, cd, sc, b, psi, G, nmat_s, chunk);
      };
      // copy slots per thread: exactly the chunks one level needs
      const int per_level = g.ny * 4 * seg_chunks;
      const int need = (per_level + threads - 1) / threads;
      auto pick = [&](auto a_tag) {
        constexpr int AA = decltype(a_tag)::value;
        auto by_u = [&](auto nst_tag) {
          constexpr int NS = decltype(nst_tag)::value;
          if (need <= 3) launch(sweep2d_rows_kernel<T, AA, NS, 3>);
          else if (need <= 6) launch(sweep2d_rows_kernel<T, AA, NS, 6>);
          else launch(sweep2d_rows_kernel<T, AA, NS, 12>);
        };
        if (NST == 2) by_u(std::integral_constant<int, 2>());
        else if (NST == 3) by_u(std::integral_constant<int, 3>());
        else if (NST == 4) by_u(std::integral_constant<int, 4>());
        else by_u(std::integral_constant<int, 6>());
      };
      if (g.a == 3) pick(std::integral_constant<int, 3>());
      else pick(std::integral_constant<int, 1>());
      return;
    }
  }
  if (g.dim == 3 && variant != 1 && err && gbar) {
    // every direction and patch at once, a grid barrier per wavefront level
    auto launch3 = [&](auto kern) -> bool {
      int per_sm = 0, dev = 0, nsm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSweep3Threads, 0) !=
              cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return false;
      }
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      int nblocks = per_sm * nsm;
      if (cudaMemsetAsync(gbar, 0, 2 * sizeof(unsigned), st) != cudaSuccess) return false;
      void* args[] = {(void*)&g, (void*)&t, (void*)&cd, (void*)&sc, (void*)&b, (void*)&psi,
                      (void*)&gbar, (void*)&err};
      if (cudaLaunchCooperativeKernel((void*)kern, dim3(nblocks), dim3(kSweep3Threads), args, 0,
                                      st) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      return true;
    };
    if (g.a == 3 ? launch3(sweep3d_grid_kernel<T, 3>) : launch3(sweep3d_grid_kernel<T, 1>)) return;
  }
  dim3 grid(sc.ntask), block(256);
  if (g.dim == 2 && g.a == 3) sweep_kernel<T, 2, 3><<<grid, block, 0, st>>>(g, t, cd, sc, b, psi);
  else if (g.dim == 2) sweep_kernel<T, 2, 1><<<grid, block, 0, st>>>(g, t, cd, sc, b, psi);
  else if (g.a == 3) sweep_kernel<T, 3, 3><<<grid, block, 0, st>>>(g, t, cd, sc, b, psi);
  else sweep_kernel<T, 3, 1><<<grid, block, 0, st>>>(g, t, cd, sc, b, psi);
}

void launch_apply_L_df(const Geom& g, const float2* aax, const float2* mang, const int* pdir,
                       const double* sigma_t, double alpha, double beta, const double* x,
                       double* y, cudaStream_t st) {
  note_launch();
  const int grid = grid_for((long long)g.C * g.P, 256);
  if (g.dim == 2 && g.a == 3)
    apply_L_df_kernel<2, 3><<<grid, 256, 0, st>>>(g, aax, mang, pdir, sigma_t, alpha, beta, x, y);
  else if (g.dim == 2)
    apply_L_df_kernel<2, 1><<<grid, 256, 0, st>>>(g, aax, mang, pdir, sigma_t, alpha, beta, x, y);
  else if (g.a == 3)
    apply_L_df_kernel<3, 3><<<grid, 256, 0, st>>>(g, aax, mang, pdir, sigma_t, alpha, beta, x, y);
  else
    apply_L_df_kernel<3, 1><<<grid, 256, 0, st>>>(g, aax, mang, pdir, sigma_t, alpha, beta, x, y);
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
                   const double* bval, const int* bkind, const double* beam,
                   const double* brange, const double* mu, const double* mf, T* f,
                   cudaStream_t st) {
  note_launch();
  const int grid = grid_for((long long)g.C * g.P, 256);
  source_kernel<T><<<grid, 256, 0, st>>>(g, w, Aw, octant, q, bval, bkind, beam, brange, mu, mf,
                                         f);
}

template <class T>
void launch_scalar_flux(long long nsdof, int nadof, const T* w, const T* psi, T* phi,
                        cudaStream_t st) {
  note_launch();
  const int grid = grid_for(nsdof * 32, 256);
  scalar_flux_kernel<T><<<grid, 256, 0, st>>>(nsdof, nadof, w, psi, phi);
}

// launch shape of the uniform-refinement transfers: threads over the coarse
// patches, blocks over bands of rows (about 8 blocks per SM in all)
static void transfer4_shape(long long nsdof, int Pc, dim3& grid, dim3& block, int& rpb) {
  const int threads = Pc >= 256 ? 256 : ((Pc + 31) / 32) * 32;
  const int gx = (Pc + threads - 1) / threads;
  long long gy = (152LL * 8 + gx - 1) / gx;
  if (gy > nsdof) gy = nsdof;
  if (gy < 1) gy = 1;
  rpb = (int)((nsdof + gy - 1) / gy);
  gy = (nsdof + rpb - 1) / rpb;
  grid = dim3((unsigned)gx, (unsigned)gy);
  block = dim3((unsigned)threads);
}
static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <class T>
void launch_restrict(long long nsdof, int Pc, int a, int nadof_f, int nadof_c, const int* cbeg,
                     const int* cend, const T* blk, const T* rf, T* rc, bool uniform4,
                     cudaStream_t st) {
  note_launch();
  if (uniform4 && a == 3 && aligned16(rf)) {
    dim3 grid, block;
    int rpb;
    transfer4_shape(nsdof, Pc, grid, block, rpb);
    restrict4_kernel<T><<<grid, block, 0, st>>>(nsdof, Pc, rpb, blk, rf, rc);
    return;
  }
  const int grid = grid_for(nsdof * Pc, 256);
  restrict_kernel<T><<<grid, 256, 0, st>>>(nsdof, Pc, a, nadof_f, nadof_c, cbeg, cend, blk, rf,
                                           rc);
}

template <class T>
void launch_prolong(long long nsdof, int Pf, int a, int nadof_f, int nadof_c, const int* parent,
                    const T* blk, const T* xc, T* xf, bool uniform4, cudaStream_t st) {
  note_launch();
  if (uniform4 && a == 3 && aligned16(xf) && Pf % 4 == 0) {
    dim3 grid, block;
    int rpb;
    transfer4_shape(nsdof, Pf / 4, grid, block, rpb);
    prolong4_kernel<T><<<grid, block, 0, st>>>(nsdof, Pf / 4, rpb, blk, xc, xf);
    return;
  }
  const int grid = grid_for(nsdof * Pf, 256);
  prolong_kernel<T><<<grid, 256, 0, st>>>(nsdof, Pf, a, nadof_f, nadof_c, parent, blk, xc, xf);
}

#define AMGT_INST(T)                                                                          \
  template void launch_sweep<T>(const Geom&, const LevelDev<T>&, const CellData&,             \
                                const Schedule&, const T*, T*, int, int, int, int, int,       \
                                int*, int, unsigned*, cudaStream_t);                          \
  template void launch_apply_L<T>(const Geom&, const LevelDev<T>&, const CellData&, T, T,     \
                                  const T*, T*, cudaStream_t);                                \
  template void launch_source<T>(const Geom&, const T*, const T*, const int*, const double*,  \
                                 const double*, const int*, const double*, const double*,     \
                                 const double*, const double*, T*, cudaStream_t);             \
  template void launch_scalar_flux<T>(long long, int, const T*, const T*, T*, cudaStream_t);  \
  template void launch_restrict<T>(long long, int, int, int, int, const int*, const int*,     \
                                   const T*, const T*, T*, bool, cudaStream_t);               \
  template void launch_prolong<T>(long long, int, int, int, int, const int*, const T*,        \
                                  const T*, T*, bool, cudaStream_t);
AMGT_INST(double)
AMGT_INST(float)
#undef AMGT_INST

}  // namespace amgt
