// Row-pipelined coarse Gauss-Seidel (Sec. 4.2), the same iteration as the
// direction-blocked kernels of kernels_gs.cu: for every sweep, every sweep
// direction d in index order and every cell c in the direction's upwind order,
//
//   x_d   = Tinv_d [ f_d - upwind_d + sigma_s N (X_d F Phi_c - S_dd^{L+D} x_d^old) ]
//   Phi_c += X_d^T (x_d - x_d^old)
//
// where Tinv_d = (D_d - sigma_s N (x) S_dd^{L+D})^{-1} solves the direction's
// patches of the cell in index order at once (block lower triangular).
//
// Schedule.  A row is the line of cells along x at fixed (y, z).  Each thread
// block owns a fixed set of rows for the whole launch and visits, per
// direction, its rows in the direction's wavefront order (increasing rotated
// y + z) and each row's cells in the direction's x order.  A cell's x-upwind
// values are the block's own previous cell (shared memory); its y- and z-
// upwind values come from the blocks owning the neighbouring rows through
// tagged words in global memory: each word carries one 32-bit payload and a
// tag naming the sweep that wrote it, so a reader spins (with a time limit) on
// the word itself and needs no fence or flag.  A cell's own unknowns and
// moments are touched by its owning block only, so no other ordering exists
// between blocks; there is no grid-wide barrier.  All blocks must be resident
// at once (cooperative launch).
//
// Deadlock freedom: every block visits its cells in one global order
// (sweep, direction, rotated level, x), and every wait is on a cell earlier
// in that order owned by another block, so the earliest unfinished cell can
// always proceed.  A face slot (direction, cell) is rewritten only one sweep
// later, after the writer has gone through a direction in which it waits on
// the reader's row, so no reader can miss its word.
#include <algorithm>
#include <cstdint>

#include "gs_common.cuh"
#include "kernels.cuh"

namespace amgt {

namespace {

constexpr int kRowsThreads = 384;  // 96 four-lane groups
constexpr int kRowsMaxU = 2;       // padded cell unknowns per thread
constexpr int kRowsMaxM = 8;       // cell moments per thread
// give up a face wait after this long: the block records code 5 in the
// status word and goes on; every later wait of every block then returns at once
constexpr unsigned long long kRowsWaitNs = 2000000000ULL;

using gsx::fcompress;
using gsx::V16;

__device__ __forceinline__ void st_word(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_word(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// A face value as tagged 64-bit words (tag in the high half): one word for a
// float, two for a double.
template <class T>
struct FaceWords;
template <>
struct FaceWords<float> {
  static constexpr int W = 1;
  __device__ static void put(unsigned long long* p, float v, unsigned tag) {
    st_word(p, ((unsigned long long)tag << 32) | __float_as_uint(v));
  }
  __device__ static void load(const unsigned long long* p, unsigned long long (&w)[W]) {
    w[0] = ld_word(p);
  }
  __device__ static bool ready(const unsigned long long (&w)[W], unsigned tag) {
    return (unsigned)(w[0] >> 32) == tag;
  }
  __device__ static float value(const unsigned long long (&w)[W]) {
    return __uint_as_float((unsigned)w[0]);
  }
};
template <>
struct FaceWords<double> {
  static constexpr int W = 2;
  __device__ static void put(unsigned long long* p, double v, unsigned tag) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    st_word(p, ((unsigned long long)tag << 32) | (b & 0xffffffffULL));
    st_word(p + 1, ((unsigned long long)tag << 32) | (b >> 32));
  }
  __device__ static void load(const unsigned long long* p, unsigned long long (&w)[W]) {
    w[0] = ld_word(p);
    w[1] = ld_word(p + 1);
  }
  __device__ static bool ready(const unsigned long long (&w)[W], unsigned tag) {
    return (unsigned)(w[0] >> 32) == tag && (unsigned)(w[1] >> 32) == tag;
  }
  __device__ static double value(const unsigned long long (&w)[W]) {
    return __longlong_as_double((long long)((w[0] & 0xffffffffULL) | (w[1] << 32)));
  }
};

template <class T>
struct RowsArgs {
  Geom g;
  LevelDev<T> t;
  CellData cd;
  int ndir;
  const int* dir_begin;  // [ndir] first patch of each direction
  const int* dir_end;
  int sweeps;
  const T* f;
  T* psi;
  T* mom;                // [C*s][nmom] flux moments, consistent with psi on entry
  const T* TinvT;        // [nmat][ndir][Emax (col)][Emax (row)]
  const T* SLD;          // [ndir][Jmax][Jmax]
  int Emax, Jmax, nmat, nmat_s;
  const int* rows;       // [ndir][nblocks][rpb] rows of each block, -1 padded
  int rpb;
  unsigned long long* faces;  // [dim-1][ndir][C][HS*Jmax][W] tagged words
  unsigned tag0;
  int* err;
};

template <class T, int DIM, int A>
__global__ void __launch_bounds__(kRowsThreads) coarse_gs_rows_kernel(RowsArgs<T> p) {
  constexpr int S = 1 << DIM;
  constexpr int HS = S / 2;
  constexpr int VW = V16<T>::n;
  constexpr int NF = DIM - 1;  // faces exchanged between rows: y (and z)
  constexpr int W = FaceWords<T>::W;
  const Geom& g = p.g;
  const int nm = p.t.nmom, nadof = g.nadof, nx = g.nx, ndir = p.ndir;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int qd = tid >> 2, l4 = tid & 3, NQ = NT >> 2;
  const int nb = gridDim.x, b = blockIdx.x;
  // padded shapes: a direction's J unknowns per node are stored Jv apart
  const int Jv = ((p.Jmax + VW - 1) / VW) * VW;
  const int Ev = S * Jv;
  const int Evp = gsx::pad16<T>(Ev), NMp = gsx::pad16<T>(nm), Jp = gsx::pad16<T>(Jv);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Tin = reinterpret_cast<T*>(smem_raw);                        // [nmat_s][Ev][Evp]
  T* XFr = Tin + gsx::round16((size_t)p.nmat_s * Ev * Evp, sizeof(T));  // [Jv][NMp]
  T* Xk = XFr + gsx::round16((size_t)Jv * NMp, sizeof(T));        // [nm][Jp]
  T* SLr = Xk + gsx::round16((size_t)nm * Jp, sizeof(T));         // [Jv][Jp]
  T* Ns = SLr + gsx::round16((size_t)Jv * Jp, sizeof(T));         // [S][S]
  T* rhs = Ns + gsx::round16(S * S, sizeof(T));                   // [S][Jv]
  T* xold = rhs + gsx::round16(Ev, sizeof(T));                    // [S][Jv]
  T* buf = xold + gsx::round16(Ev, sizeof(T));                    // [S][Jv]
  T* phs = buf + gsx::round16(Ev, sizeof(T));                     // [S][NMp]
  T* xfc = phs + gsx::round16((size_t)S * NMp, sizeof(T));        // [HS][Jv] x-outflow
  T* yup = xfc + gsx::round16((size_t)HS * Jv, sizeof(T));        // [NF][HS][Jv] inflow
  for (int i = tid; i < S * S; i += NT) Ns[i] = (T)g.Nmass[i];
  for (int i = tid; i < Ev; i += NT) rhs[i] = xold[i] = buf[i] = T(0);
  for (int i = tid; i < S * NMp; i += NT) phs[i] = T(0);
  const int nrow_cells = nx;
  const int* myrows = p.rows + (size_t)b * p.rpb;  // + d * nb * rpb per direction
  auto row_of = [&](int d, int ri) -> int {
    return ri < p.rpb ? myrows[(size_t)d * nb * p.rpb + ri] : -1;
  };
  auto dir_bits = [&](int d, int& n0, int& n1, int& n2) {
    if (DIM == 2) {
      n0 = (d >> 1) & 1; n1 = d & 1; n2 = 0;
    } else {
      n0 = (d >> 2) & 1; n1 = (d >> 1) & 1; n2 = d & 1;
    }
  };
  // prefetch registers for the next cell
  T pf[kRowsMaxU], px[kRowsMaxU], pm[kRowsMaxM];
  auto prefetch = [&](int d, int R, int k) {
    int n0, n1, n2;
    dir_bits(d, n0, n1, n2);
    const int ix = n0 ? nx - 1 - k : k;
    const long long c = ix + (long long)nx * R;
    const int qb = p.dir_begin[d];
    const int J = (p.dir_end[d] - qb) * A;
#pragma unroll
    for (int u = 0; u < kRowsMaxU; ++u) {
      const int pe = tid + u * NT;
      pf[u] = T(0);
      px[u] = T(0);
      if (pe < Ev) {
        const int l = pe / Jv, j = pe - l * Jv;
        if (j < J) {
          const long long gix = (c * S + l) * nadof + qb * A + j;
          pf[u] = p.f[gix];
          px[u] = __ldcg(p.psi + gix);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kRowsMaxM; ++u) {
      const int e = tid + u * NT;
      if (e < S * nm) pm[u] = __ldcg(p.mom + c * S * nm + e);
    }
  };
  long long prev_cell = -1;
  {
    const int R0 = row_of(0, 0);
    if (R0 >= 0 && p.sweeps > 0) prefetch(0, R0, 0);
  }
  for (int sw = 0; sw < p.sweeps; ++sw) {
    const unsigned tag = p.tag0 + (unsigned)sw + 1u;
    for (int d = 0; d < ndir; ++d) {
      int n0, n1, n2;
      dir_bits(d, n0, n1, n2);
      const int qb = p.dir_begin[d];
      const int J = (p.dir_end[d] - qb) * A;
      const int E = S * J;
      // stage this direction's tables (padded, zero filled)
      __syncthreads();
      for (int mt = 0; mt < p.nmat_s; ++mt) {
        const T* src = p.TinvT + ((size_t)mt * ndir + d) * p.Emax * p.Emax;  // [col][row]
        T* dst = Tin + (size_t)mt * Ev * Evp;
        for (int i = tid; i < Ev * Ev; i += NT) {
          const int cp = i / Ev, rp = i - cp * Ev;  // padded column, row
          const int lc = cp / Jv, jc = cp - lc * Jv, lr = rp / Jv, jr = rp - lr * Jv;
          dst[(size_t)rp * Evp + cp] =
              (jc < J && jr < J) ? src[(size_t)(lc * J + jc) * p.Emax + lr * J + jr] : T(0);
        }
      }
      for (int i = tid; i < Jv * NMp; i += NT) {
        const int j = i / NMp, kk = i - j * NMp;
        XFr[i] = (j < J && kk < nm) ? p.t.XFt[(long long)kk * nadof + qb * A + j] : T(0);
      }
      for (int i = tid; i < nm * Jp; i += NT) {
        const int kk = i / Jp, j = i - kk * Jp;
        Xk[i] = j < J ? p.t.X[(long long)(qb * A + j) * nm + kk] : T(0);
      }
      for (int i = tid; i < Jv * Jp; i += NT) {
        const int j = i / Jp, j2 = i - j * Jp;
        SLr[i] = (j < J && j2 < J) ? p.SLD[((size_t)d * p.Jmax + j) * p.Jmax + j2] : T(0);
      }
      __syncthreads();
      for (int ri = 0;; ++ri) {
        const int R = row_of(d, ri);
        if (R < 0) break;
        const int iy = R % g.ny, iz = R / g.ny;
        const int jy = n1 ? g.ny - 1 - iy : iy;
        const int jz = n2 ? g.nz - 1 - iz : iz;
        for (int k = 0; k < nrow_cells; ++k) {
          const int ix = n0 ? nx - 1 - k : k;
          const long long c = ix + (long long)nx * R;
          const int mat = p.cd.mat[c];
          const T sig_s = (T)p.cd.sigma_s[c];
          // ---- A: the cell's data into shared memory; first look at the faces
#pragma unroll
          for (int u = 0; u < kRowsMaxU; ++u) {
            const int pe = tid + u * NT;
            if (pe < Ev) {
              rhs[pe] = pf[u];
              xold[pe] = px[u];
            }
          }
          if (c != prev_cell) {
#pragma unroll
            for (int u = 0; u < kRowsMaxM; ++u) {
              const int e = tid + u * NT;
              if (e < S * nm) {
                const int l = e / nm;
                phs[l * NMp + (e - l * nm)] = pm[u];
              }
            }
          }
          // face words this thread waits for: (axis, face node, unknown)
          const int npoll = NF * HS * J;
          bool need = false;
          const unsigned long long* wp = nullptr;
          unsigned long long fw[W];
          int pa = 0, pjn = 0, pj = 0;
          if (tid < npoll) {
            pa = tid / (HS * J);
            const int rem = tid - pa * HS * J;
            pjn = rem / J;
            pj = rem - pjn * J;
            const int jr = pa == 0 ? jy : jz;
            if (jr > 0) {
              const int own = pa == 0 ? n1 : n2;
              const long long strd = pa == 0 ? (long long)nx : (long long)nx * g.ny;
              const long long cn = c + (own ? strd : -strd);
              wp = p.faces + ((((size_t)pa * ndir + d) * g.C + cn) * HS * p.Jmax +
                              (size_t)pjn * J + pj) * W;
              need = true;
              FaceWords<T>::load(wp, fw);
            }
          }
          __syncthreads();
          // the next cell of this block's sequence into registers
          {
            int d2 = d, ri2 = ri, k2 = k + 1, sw2 = sw;
            bool more = true;
            if (k2 >= nrow_cells) {
              k2 = 0;
              ++ri2;
              if (row_of(d2, ri2) < 0) {
                ri2 = 0;
                if (++d2 >= ndir) {
                  d2 = 0;
                  more = ++sw2 < p.sweeps;
                }
              }
            }
            if (more) prefetch(d2, row_of(d2, ri2), k2);
          }
          // ---- B: buf = X_d F Phi - S_dd^{L+D} x_old (four lanes per unknown)
          for (int base = 0; base < Ev; base += NQ) {
            const int pe = base + qd;
            const int l = pe / Jv, j = pe - l * Jv;
            const bool valid = pe < Ev && j < J;
            T a = T(0);
            if (valid) {
              const T* xr = XFr + j * NMp;
              const T* ph = phs + l * NMp;
              for (int ch = l4 * VW; ch < NMp; ch += 4 * VW) a += V16<T>::dot(xr + ch, ph + ch);
              const T* sl = SLr + j * Jp;
              const T* xo = xold + l * Jv;
              for (int ch = l4 * VW; ch < Jv; ch += 4 * VW) a -= V16<T>::dot(sl + ch, xo + ch);
            }
            a += __shfl_xor_sync(0xffffffffu, a, 1);
            a += __shfl_xor_sync(0xffffffffu, a, 2);
            if (pe < Ev && l4 == 0) buf[pe] = valid ? a : T(0);
          }
          // the upwind rows' face words
          if (need) {
            if (!FaceWords<T>::ready(fw, tag)) {
              const unsigned long long t0 = gsx::now_ns();
              unsigned it = 0;
              do {
                FaceWords<T>::load(wp, fw);
                if ((++it & 63u) == 0) {
                  // after any block gave up, the others stop waiting too
                  if (gsx::now_ns() - t0 > kRowsWaitNs) atomicExch(p.err, 5);
                  if (*reinterpret_cast<volatile int*>(p.err) != 0) break;
                }
              } while (!FaceWords<T>::ready(fw, tag));
            }
            yup[(pa * HS + pjn) * Jv + pj] = FaceWords<T>::value(fw);
          }
          __syncthreads();
          // ---- C: rhs = f - upwind + sigma_s N buf
          for (int pe = tid; pe < Ev; pe += NT) {
            const int l = pe / Jv, j = pe - l * Jv;
            if (j >= J) continue;
            const int q = qb + j / A, m = j % A, jb = (j / A) * A;
            T val = rhs[pe];
#pragma unroll
            for (int xi = 0; xi < DIM; ++xi) {
              const int own = xi == 0 ? n0 : (xi == 1 ? n1 : n2);
              const int jr = xi == 0 ? k : (xi == 1 ? jy : jz);
              if (jr == 0 || ((l >> xi) & 1) != own) continue;
              const T* up = xi == 0 ? xfc : yup + (size_t)(xi - 1) * HS * Jv;
              const T* An = p.t.Aax + ((size_t)q * 3 + xi) * A * A + m * A;
              const int jp = fcompress(l, xi);
              T acc = T(0);
#pragma unroll
              for (int jn = 0; jn < HS; ++jn) {
                T sacc = T(0);
#pragma unroll
                for (int dd = 0; dd < A; ++dd) sacc += __ldg(An + dd) * up[jn * Jv + jb + dd];
                acc += T(g.facemass[xi][jp][jn]) * sacc;
              }
              val -= (own ? T(1) : T(-1)) * acc;
            }
            T mix = T(0);
#pragma unroll
            for (int i = 0; i < S; ++i) mix += Ns[l * S + i] * buf[i * Jv + j];
            rhs[pe] = val + sig_s * mix;
          }
          __syncthreads();
          // ---- D: x_new = Tinv rhs (four lanes per row); outputs
          for (int base = 0; base < Ev; base += NQ) {
            const int pe = base + qd;
            const int l = pe / Jv, j = pe - l * Jv;
            const bool valid = pe < Ev && j < J;
            T a = T(0);
            if (valid) {
              if (mat < p.nmat_s) {
                const T* row = Tin + ((size_t)mat * Ev + pe) * Evp;
                for (int ch = l4 * VW; ch < Ev; ch += 4 * VW) a += V16<T>::dot(row + ch, rhs + ch);
              } else {
                const T* col = p.TinvT + ((size_t)mat * ndir + d) * p.Emax * p.Emax + l * J + j;
                for (int cc = l4; cc < E; cc += 4) {
                  const int lc = cc / J;
                  a += __ldg(col + (size_t)cc * p.Emax) * rhs[lc * Jv + (cc - lc * J)];
                }
              }
            }
            a += __shfl_xor_sync(0xffffffffu, a, 1);
            a += __shfl_xor_sync(0xffffffffu, a, 2);
            if (pe < Ev && l4 == 0) {
              if (valid) {
                p.psi[(c * S + l) * nadof + qb * A + j] = a;
                buf[pe] = a - xold[pe];
                if (((l & 1) ^ n0) == 1) xfc[fcompress(l, 0) * Jv + j] = a;
#pragma unroll
                for (int xi = 1; xi < DIM; ++xi) {
                  const int own = xi == 1 ? n1 : n2;
                  const int jr = xi == 1 ? jy : jz;
                  const int nn = xi == 1 ? g.ny : g.nz;
                  if (((l >> xi) & 1) == own || jr == nn - 1) continue;
                  unsigned long long* wq =
                      p.faces + ((((size_t)(xi - 1) * ndir + d) * g.C + c) * HS * p.Jmax +
                                 (size_t)fcompress(l, xi) * J + j) * W;
                  FaceWords<T>::put(wq, a, tag);
                }
              } else {
                buf[pe] = T(0);
              }
            }
          }
          __syncthreads();
          // ---- E: Phi_c += X_d^T delta
          for (int base = 0; base < S * nm; base += NQ) {
            const int e = base + qd;
            const int l = e / nm, kk = e - l * nm;
            T a = T(0);
            if (e < S * nm) {
              const T* xr = Xk + kk * Jp;
              const T* dl = buf + l * Jv;
              for (int ch = l4 * VW; ch < Jv; ch += 4 * VW) a += V16<T>::dot(xr + ch, dl + ch);
            }
            a += __shfl_xor_sync(0xffffffffu, a, 1);
            a += __shfl_xor_sync(0xffffffffu, a, 2);
            if (e < S * nm && l4 == 0) {
              const T v = phs[l * NMp + kk] + a;
              phs[l * NMp + kk] = v;
              p.mom[c * S * nm + e] = v;
            }
          }
          prev_cell = c;
          __syncthreads();
        }
      }
    }
  }
}

template <class T>
size_t rows_smem_bytes(int nmat_s, int Emax, int Jmax, int nm, int s) {
  const int vw = 16 / (int)sizeof(T);
  const int Jv = ((Jmax + vw - 1) / vw) * vw, Ev = s * Jv;
  const int Evp = gsx::pad16<T>(Ev), NMp = gsx::pad16<T>(nm), Jp = gsx::pad16<T>(Jv);
  (void)Emax;
  const size_t e = gsx::round16((size_t)nmat_s * Ev * Evp, sizeof(T)) +
                   gsx::round16((size_t)Jv * NMp, sizeof(T)) + gsx::round16((size_t)nm * Jp, sizeof(T)) +
                   gsx::round16((size_t)Jv * Jp, sizeof(T)) + gsx::round16((size_t)s * s, sizeof(T)) +
                   3 * gsx::round16((size_t)Ev, sizeof(T)) + gsx::round16((size_t)s * NMp, sizeof(T)) +
                   gsx::round16((size_t)(s / 2) * Jv, sizeof(T)) +
                   gsx::round16((size_t)2 * (s / 2) * Jv, sizeof(T));
  return e * sizeof(T);
}

template <class T, int DIM, int A>
cudaError_t rows_launch(const RowsArgs<T>& a, int nblocks, size_t smem, cudaStream_t st) {
  auto kern = coarse_gs_rows_kernel<T, DIM, A>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((void*)kern, dim3(nblocks), dim3(kRowsThreads), args, smem, st);
}

template <class T, int DIM, int A>
int rows_max_blocks(size_t smem) {
  auto kern = coarse_gs_rows_kernel<T, DIM, A>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRowsThreads, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * nsm;
}

}  // namespace

template <class T>
int coarse_gs_rows_plan(const Geom& g, int nmat, int Emax, int Jmax, int nmom, int* nmat_s,
                        size_t* smem) {
  const int vw = 16 / (int)sizeof(T);
  const int Jv = ((Jmax + vw - 1) / vw) * vw, Ev = g.s * Jv;
  if (g.a != 1 && g.a != 3) return 0;
  if (Ev > kRowsMaxU * kRowsThreads || g.s * nmom > kRowsMaxM * kRowsThreads ||
      (g.dim - 1) * (g.s / 2) * Jmax > kRowsThreads || g.nx < 1)
    return 0;
  int ns = nmat;
  while (ns > 0 && rows_smem_bytes<T>(ns, Emax, Jmax, nmom, g.s) > 200 * 1024) --ns;
  const size_t bytes = rows_smem_bytes<T>(ns, Emax, Jmax, nmom, g.s);
  if (bytes > 200 * 1024) return 0;
  int nb;
  if (g.dim == 2) nb = g.a == 3 ? rows_max_blocks<T, 2, 3>(bytes) : rows_max_blocks<T, 2, 1>(bytes);
  else nb = g.a == 3 ? rows_max_blocks<T, 3, 3>(bytes) : rows_max_blocks<T, 3, 1>(bytes);
  const int nrows = g.ny * g.nz;
  nb = std::min(nb, nrows);
  *nmat_s = ns;
  *smem = bytes;
  return nb;
}

template <class T>
int launch_coarse_gs_rows(const Geom& g, const LevelDev<T>& t, const CellData& cd, int ndir,
                          const int* dir_begin, const int* dir_end, int sweeps, const T* f,
                          T* phi, T* mom, const T* TinvT, const T* SLD, int Emax, int Jmax,
                          int nmat, int nmat_s, size_t smem, const int* rows, int nblocks,
                          int rpb, unsigned long long* faces, unsigned tag0, int* err,
                          cudaStream_t st) {
  RowsArgs<T> a{g, t, cd, ndir, dir_begin, dir_end, sweeps, f, phi, mom, TinvT, SLD,
                Emax, Jmax, nmat, nmat_s, rows, rpb, faces, tag0, err};
  cudaError_t e;
  if (g.dim == 2) e = g.a == 3 ? rows_launch<T, 2, 3>(a, nblocks, smem, st) : rows_launch<T, 2, 1>(a, nblocks, smem, st);
  else e = g.a == 3 ? rows_launch<T, 3, 3>(a, nblocks, smem, st) : rows_launch<T, 3, 1>(a, nblocks, smem, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  note_launch();
  return 0;
}

template int coarse_gs_rows_plan<float>(const Geom&, int, int, int, int, int*, size_t*);
template int coarse_gs_rows_plan<double>(const Geom&, int, int, int, int, int*, size_t*);
template int launch_coarse_gs_rows<float>(const Geom&, const LevelDev<float>&, const CellData&, int,
                                          const int*, const int*, int, const float*, float*,
                                          float*, const float*, const float*, int, int, int, int,
                                          size_t, const int*, int, int, unsigned long long*,
                                          unsigned, int*, cudaStream_t);
template int launch_coarse_gs_rows<double>(const Geom&, const LevelDev<double>&, const CellData&,
                                           int, const int*, const int*, int, const double*,
                                           double*, double*, const double*, const double*, int,
                                           int, int, int, size_t, const int*, int, int,
                                           unsigned long long*, unsigned, int*, cudaStream_t);

}  // namespace amgt
