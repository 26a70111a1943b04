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
// Dense form.  Where the cell's angular unknowns are fewer than twice its
// moments, the moments are not kept: with S_f = X F X^T (one moment shape)
//
//   X_d F Phi_c - S_dd^{L+D} x_d^old = M_d x_c,   M_d = S_f[d rows] - S_dd^{L+D}
//
// (S_dd^{L+D} subtracted in the direction's own columns), a product with the
// cell's current unknowns x_c over all directions; the moment update goes.
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

constexpr int kRowsMaxThreads = 512;
constexpr int kRowsMaxU = 2;  // padded cell unknowns per thread
constexpr int kRowsMaxM = 8;  // cell moments per thread
// prefetch register shapes (unknowns, moments per thread) of the kernel
// instantiations: a prefetched value spilled to local memory would make the
// prefetch wait for its load, so each launch takes the smallest shape that
// holds its cell
__host__ __device__ inline int rows_shape(int Ev, int Snm, int nt) {
  if (Ev <= nt && Snm <= nt) return 0;       // 1, 1
  if (Ev <= 2 * nt && Snm <= 2 * nt) return 1;  // 2, 2
  return 2;                                     // 2, 8
}
// give up a face wait after this long: the block records code 5 in the
// status word and goes on; every later wait of every block then returns at once
constexpr unsigned long long kRowsWaitNs = 2000000000ULL;

using gsx::fcompress;
using gsx::V16;

// Row stride (elements of T) for tables read by four-lane groups, each lane
// taking every fourth 16-byte chunk of a row: a stride of 64 bytes modulo 128
// puts the two rows read by one quarter warp on disjoint banks.
template <class T>
__host__ __device__ inline int qpad(int n) {
  const int vw = 16 / (int)sizeof(T);
  int p = ((n + vw - 1) / vw) * vw;
  while ((p * (int)sizeof(T)) % 128 != 64) p += vw;
  return p;
}

// Shared-memory layout of one block (byte offsets, 16-byte aligned).
template <class T>
struct RowsLayout {
  int Jv, Ev, Evp, NMp, Jp, Eyl, Wp;
  size_t o_Tin, o_XFr, o_Xk, o_SLr, o_Ns, o_Ad, o_lj, o_lk, o_rhs, o_xold, o_buf, o_phs, o_xfc,
      o_yup, o_Tg, o_W, o_y0, bytes;
  // gbuf: elements of one prefetch buffer for a block inverse that is not
  // staged (0: read those from global memory)
  // nm: moments per node, or in the dense form the angular unknowns (the
  // cell's x_c takes the moments' place and X_d, S_dd^{L+D} are not staged)
  __host__ __device__ RowsLayout(int nmat_s, int Jmax, int nm, int S, int dim, int A, int ndir,
                                 int gbuf, bool dense) {
    const int vw = 16 / (int)sizeof(T);
    Jv = ((Jmax + vw - 1) / vw) * vw;
    Ev = S * Jv;
    Evp = qpad<T>(Ev);
    NMp = qpad<T>(nm);
    Jp = qpad<T>(Jv);
    Eyl = (dim - 1) * (S / 2) * Jv;  // inflow unknowns from the other rows' blocks
    Wp = qpad<T>(Eyl);
    size_t o = 0;
    auto take = [&](size_t nbytes) {
      const size_t at = o;
      o += (nbytes + 15) / 16 * 16;
      return at;
    };
    const size_t t = sizeof(T);
    o_Tin = take((size_t)nmat_s * Ev * Evp * t);
    o_XFr = take((size_t)Jv * NMp * t);
    o_Xk = take(dense ? 0 : (size_t)Jv * NMp * t);
    o_SLr = take(dense ? 0 : (size_t)Jv * Jp * t);
    o_Ns = take((size_t)S * S * t);
    o_Ad = take((size_t)Jmax * dim * A * t);   // [patch][axis][A][A]
    o_lj = take((size_t)ndir * Ev * sizeof(int));
    o_lk = take((size_t)S * nm * sizeof(int));
    o_rhs = take((size_t)Ev * t);
    o_xold = take((size_t)Ev * t);
    o_buf = take((size_t)2 * Ev * t);
    o_phs = take((size_t)2 * S * NMp * t);
    o_xfc = take((size_t)(S / 2) * Jv * t);
    o_yup = take((size_t)(dim - 1) * (S / 2) * Jv * t);
    o_Tg = take((size_t)2 * gbuf * t);
    o_W = take((size_t)nmat_s * Ev * Wp * t);
    o_y0 = take((size_t)Ev * t);
    bytes = o;
  }
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
// all but the most recent group complete
__device__ __forceinline__ void cp_async_wait_prior() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

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
  const T* Sf;           // [nadof][nadof] S_f (dense form)
  int dense;             // 1: dense form (mom unused, x_c read from psi)
  int Emax, Jmax, nmat, nmat_s;
  int gbuf;              // > 0: inverses of unstaged materials prefetched into shared memory
  const int* rows;       // [ndir][nblocks][rpb] rows of each block, -1 padded
  int rpb;
  unsigned long long* faces;  // [dim-1][ndir][C][HS*Jmax][W] tagged words
  unsigned tag0;
  int* err;
};

// Per-direction staging of the tables into shared memory (padded, zero
// filled), by the block's NT threads.  Block inverses of the staged materials:
// Tin[mt][row][col] over the padded unknowns (l Jv + j).
template <class T>
__device__ void stage_tinv(const RowsArgs<T>& p, T* Tin, int d, int J, int Jv, int Ev, int Evp,
                           int tid, int NT) {
  for (int mt = 0; mt < p.nmat_s; ++mt) {
    const T* src = p.TinvT + ((size_t)mt * p.ndir + d) * p.Emax * p.Emax;  // [col][row]
    T* dst = Tin + (size_t)mt * Ev * Evp;
    for (int i = tid; i < Ev * Ev; i += NT) {
      const int cp = i / Ev, rp = i - cp * Ev;  // padded column, row
      const int lc = cp / Jv, jc = cp - lc * Jv, lr = rp / Jv, jr = rp - lr * Jv;
      dst[(size_t)rp * Evp + cp] =
          (jc < J && jr < J) ? src[(size_t)(lc * J + jc) * p.Emax + lr * J + jr] : T(0);
    }
  }
}
// M_d = S_f[d rows] - S_dd^{L+D} in the direction's own columns: [Jv][NMp]
template <class T>
__device__ void stage_md(const RowsArgs<T>& p, T* Md, int d, int q0, int J, int Jv, int NMp,
                         int nadof, int tid, int NT) {
  for (int i = tid; i < Jv * NMp; i += NT) {
    const int j = i / NMp, kk = i - j * NMp;
    T v = T(0);
    if (j < J && kk < nadof) {
      v = p.Sf[(long long)(q0 + j) * nadof + kk];
      const int j2 = kk - q0;
      if (j2 >= 0 && j2 < J) v -= p.SLD[((size_t)d * p.Jmax + j) * p.Jmax + j2];
    }
    Md[i] = v;
  }
}
// A^xi of the direction's patches: Ad[patch][axis][A][A]
template <class T, int DIM, int A>
__device__ void stage_ad(const RowsArgs<T>& p, T* Ad, int qb, int J, int tid, int NT) {
  for (int i = tid; i < (J / A) * DIM * A * A; i += NT) {
    const int jq = i / (DIM * A * A), rem = i - jq * DIM * A * A;
    const int xi = rem / (A * A), e = rem - xi * A * A;
    Ad[i] = p.t.Aax[((size_t)(qb + jq) * 3 + xi) * A * A + e];
  }
}
// W[(lr, jr)][(axis, jn, jq A + dd)] = sum over the inflow-face nodes l and m
// of Tinv[(lr, jr)][(l, jq A + m)] U, with U the coupling of the rhs of
// (l, jq A + m) to the upwind face value (jn, jq A + dd) as in the rhs
// assembly; reads the staged Tin and Ad (a barrier after their staging)
template <class T, int DIM, int A>
__device__ void stage_w(const RowsArgs<T>& p, const T* Tin, const T* Ad, T* Wl, const int* lj_d,
                        int J, int Jv, int Ev, int Evp, int Eyl, int Wp, int n1, int n2, int tid,
                        int NT) {
  constexpr int S = 1 << DIM, HS = S / 2;
  for (int i = tid; i < p.nmat_s * Ev * Eyl; i += NT) {
    const int mt = i / (Ev * Eyl);
    const int rem = i - mt * Ev * Eyl;
    const int pe = rem / Eyl, ey = rem - pe * Eyl;
    const int xi = 1 + ey / (HS * Jv);
    const int jn = (ey / Jv) % HS, jc = ey % Jv;
    T w = T(0);
    if (lj_d[pe] >= 0 && jc < J) {
      const int own = xi == 1 ? n1 : n2;
      const int jq = jc / A, dd = jc - jq * A;
      const T sg = own ? T(-1) : T(1);
      const T* trow = Tin + ((size_t)mt * Ev + pe) * Evp;
#pragma unroll
      for (int l = 0; l < S; ++l) {
        if (((l >> xi) & 1) != own) continue;
        const T fm = sg * T(p.g.facemass[xi][fcompress(l, xi)][jn]);
#pragma unroll
        for (int m = 0; m < A; ++m)
          w += trow[l * Jv + jq * A + m] * fm * Ad[((size_t)jq * DIM + xi) * A * A + m * A + dd];
      }
    }
    Wl[((size_t)mt * Ev + pe) * Wp + ey] = w;
  }
}

template <class T, int DIM, int A, int UM, int MM>
__global__ void __launch_bounds__(kRowsMaxThreads, 1) coarse_gs_rows_kernel(RowsArgs<T> p) {
  constexpr int S = 1 << DIM;
  constexpr int HS = S / 2;
  constexpr int VW = V16<T>::n;
  constexpr int NF = DIM - 1;  // faces exchanged between rows: y (and z)
  constexpr int W = FaceWords<T>::W;
  const Geom& g = p.g;
  const int nadof = g.nadof, nx = g.nx, ndir = p.ndir;
  const bool dense = p.dense != 0;
  const int nm = dense ? nadof : p.t.nmom;  // values of the cell vector per node
  const int tid = threadIdx.x, NT = blockDim.x;
  const int qd = tid >> 2, l4 = tid & 3, NQ = NT >> 2;
  const int nb = gridDim.x, b = blockIdx.x;
  const RowsLayout<T> Ly(p.nmat_s, p.Jmax, nm, S, DIM, A, ndir, p.gbuf, dense);
  // padded shapes: a direction's J unknowns per node are stored Jv apart
  const int Jv = Ly.Jv, Ev = Ly.Ev, Evp = Ly.Evp, NMp = Ly.NMp, Jp = Ly.Jp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Tin = reinterpret_cast<T*>(smem_raw + Ly.o_Tin);    // [nmat_s][Ev][Evp]
  T* XFr = reinterpret_cast<T*>(smem_raw + Ly.o_XFr);    // [Jv][NMp]  (diag(f) X_d^T)^T, or M_d
  T* Xd = reinterpret_cast<T*>(smem_raw + Ly.o_Xk);      // [Jv][NMp]  X_d (row j: unknown j's moments)
  T* SLr = reinterpret_cast<T*>(smem_raw + Ly.o_SLr);    // [Jv][Jp]   S_dd^{L+D}
  T* Ns = reinterpret_cast<T*>(smem_raw + Ly.o_Ns);      // [S][S]
  T* Ad = reinterpret_cast<T*>(smem_raw + Ly.o_Ad);      // [patch][axis][A][A]
  int* slj = reinterpret_cast<int*>(smem_raw + Ly.o_lj); // [ndir][Ev] l<<16|j, -1 past J
  int* slk = reinterpret_cast<int*>(smem_raw + Ly.o_lk); // [S*nm] l<<16|k
  T* rhs = reinterpret_cast<T*>(smem_raw + Ly.o_rhs);    // [S][Jv]
  T* xold = reinterpret_cast<T*>(smem_raw + Ly.o_xold);  // [S][Jv]
  T* bufs = reinterpret_cast<T*>(smem_raw + Ly.o_buf);   // [2][S][Jv] by cell parity
  T* phss = reinterpret_cast<T*>(smem_raw + Ly.o_phs);   // [2][S][NMp] Phi_c (or x_c) by cell parity
  T* xfc = reinterpret_cast<T*>(smem_raw + Ly.o_xfc);    // [HS][Jv] x-outflow of the last cell
  T* yup = reinterpret_cast<T*>(smem_raw + Ly.o_yup);    // [NF][HS][Jv] y/z inflow
  T* Tg = reinterpret_cast<T*>(smem_raw + Ly.o_Tg);      // [2][Emax (col)][Emax (row)]
  // Tinv U for the y/z inflow of staged materials: x = Tinv rhs0 + W yup, so
  // the block solve runs before the other rows' face values arrive
  T* Wl = reinterpret_cast<T*>(smem_raw + Ly.o_W);       // [nmat_s][Ev][Wp]
  T* y0 = reinterpret_cast<T*>(smem_raw + Ly.o_y0);      // [Ev] Tinv rhs0
  const int Eyl = Ly.Eyl, Wp = Ly.Wp;
  for (int i = tid; i < Eyl; i += NT) yup[i] = T(0);  // padding stays zero
  // first patch of each direction, kept on chip: the prefetch computes its
  // addresses from it, and a global load there would stall every cell
  __shared__ int sdb[8];
  if (tid < ndir) sdb[tid] = p.dir_begin[tid];
  for (int i = tid; i < S * S; i += NT) Ns[i] = (T)g.Nmass[i];
  for (int i = tid; i < 2 * Ev; i += NT) bufs[i] = T(0);
  for (int i = tid; i < 2 * S * NMp; i += NT) phss[i] = T(0);
  for (int i = tid; i < ndir * Ev; i += NT) {
    const int d = i / Ev, pe = i - d * Ev;
    const int J = (p.dir_end[d] - p.dir_begin[d]) * A;
    const int l = pe / Jv, j = pe - l * Jv;
    slj[i] = j < J ? (l << 16) | j : -1;
  }
  for (int i = tid; i < S * nm; i += NT) slk[i] = ((i / nm) << 16) | (i % nm);
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
  __syncthreads();
  long long kc = 0;     // cells solved by this block (buffer parity)
  // prefetch registers for the next cell
  T pf[UM], px[UM], pm[MM];
  int pmat = 0;
  T psig = T(0);
  long long c_next = -1;
  auto prefetch = [&](int d, int R, int k) {
    int n0, n1, n2;
    dir_bits(d, n0, n1, n2);
    const int ix = n0 ? nx - 1 - k : k;
    const long long c = ix + (long long)nx * R;
    c_next = c;
    const int qa = sdb[d] * A;
#pragma unroll
    for (int u = 0; u < UM; ++u) {
      const int pe = tid + u * NT;
      pf[u] = T(0);
      px[u] = T(0);
      if (pe < Ev) {
        const int lj = slj[d * Ev + pe];
        if (lj >= 0) {
          const long long gix = (c * S + (lj >> 16)) * nadof + qa + (lj & 0xffff);
          pf[u] = p.f[gix];
          px[u] = __ldcg(p.psi + gix);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < MM; ++u) {
      const int e = tid + u * NT;
      if (e < S * nm) pm[u] = __ldcg((dense ? p.psi : p.mom) + c * S * nm + e);
    }
    pmat = p.cd.mat[c];
    // sigma_s in the kernel's precision: a conversion here would wait for the
    // load and stall the prefetch
    if constexpr (sizeof(T) == 4) psig = p.cd.sigma_s32[c];
    else psig = p.cd.sigma_s[c];
    // the block inverse of an unstaged material into the free buffer (pmat is
    // only waited for when such materials exist)
    if (p.gbuf > 0) {
      if (pmat >= p.nmat_s) {
        const char* src = reinterpret_cast<const char*>(
            p.TinvT + ((size_t)pmat * ndir + d) * p.Emax * p.Emax);
        char* dst = reinterpret_cast<char*>(Tg + (size_t)((kc + 1) & 1) * p.gbuf);
        const int nchunk = p.Emax * p.Emax * (int)sizeof(T) / 16;
        for (int i = tid; i < nchunk; i += NT) cp_async16(dst + 16 * i, src + 16 * i);
      }
    }
  };
  // Phi_c += X_d^T delta for the cell `cp` whose delta is in buffer `slot`;
  // also into the other buffer when the next cell is the same cell.  One
  // thread per moment (l, k): it reads column k of X_d (consecutive threads,
  // consecutive k: no bank conflicts) and the node's delta as 16-byte chunks
  // (one address per warp: a broadcast); the stores to mom are coalesced.
  // In the dense form only a next cell equal to this one needs its x_c: the
  // old one with direction dp's block advanced by delta.
  auto update_moments = [&](long long cp, int slot, bool next_same, int dp) {
    const T* bf = bufs + (size_t)slot * Ev;
    T* ph = phss + (size_t)slot * S * NMp;
    T* ph2 = phss + (size_t)(slot ^ 1) * S * NMp;
    if (dense) {
      if (!next_same) return;
      const int q0 = sdb[dp] * A, Jd = (p.dir_end[dp] - sdb[dp]) * A;
      for (int e = tid; e < S * nm; e += NT) {
        const int lk = slk[e];
        const int o = (lk >> 16) * NMp + (lk & 0xffff);
        const int jd = (lk & 0xffff) - q0;
        ph2[o] = ph[o] + (jd >= 0 && jd < Jd ? bf[(lk >> 16) * Jv + jd] : T(0));
      }
      return;
    }
    for (int e = tid; e < S * nm; e += NT) {
      const int lk = slk[e];
      const int o = (lk >> 16) * NMp + (lk & 0xffff);
      const T* xc = Xd + (lk & 0xffff);
      const T* dl = bf + (lk >> 16) * Jv;
      T a0 = T(0), a1 = T(0);
      for (int j = 0; j < Jv; j += VW) {
        if constexpr (VW == 4) {
          const float4 dv = *reinterpret_cast<const float4*>(dl + j);
          a0 += xc[(size_t)j * NMp] * dv.x;
          a1 += xc[(size_t)(j + 1) * NMp] * dv.y;
          a0 += xc[(size_t)(j + 2) * NMp] * dv.z;
          a1 += xc[(size_t)(j + 3) * NMp] * dv.w;
        } else {
          const double2 dv = *reinterpret_cast<const double2*>(dl + j);
          a0 += xc[(size_t)j * NMp] * dv.x;
          a1 += xc[(size_t)(j + 1) * NMp] * dv.y;
        }
      }
      const T v = ph[o] + (a0 + a1);
      p.mom[cp * S * nm + e] = v;
      if (next_same) ph2[o] = v;
    }
  };
  {
    const int R0 = row_of(0, 0);
    kc = -1;  // the first cell's inverse goes to buffer 0
    if (R0 >= 0 && p.sweeps > 0) prefetch(0, R0, 0);
    cp_async_commit_group();
    kc = 0;
  }
  long long last = -1;  // last cell solved
  bool pend = false;    // its moment update is still to be done
  for (int sw = 0; sw < p.sweeps; ++sw) {
    const unsigned tag = p.tag0 + (unsigned)sw + 1u;
    for (int d = 0; d < ndir; ++d) {
      int n0, n1, n2;
      dir_bits(d, n0, n1, n2);
      const int qb = p.dir_begin[d];
      const int J = (p.dir_end[d] - qb) * A;
      const int E = S * J;
      const int* lj_d = slj + d * Ev;
      // the pending moment update uses the previous direction's tables
      __syncthreads();
      if (pend) update_moments(last, (int)((kc - 1) & 1), c_next == last, d > 0 ? d - 1 : ndir - 1);
      pend = false;
      __syncthreads();
      // stage this direction's tables (padded, zero filled)
      stage_tinv(p, Tin, d, J, Jv, Ev, Evp, tid, NT);
      if (dense) {
        stage_md(p, XFr, d, qb * A, J, Jv, NMp, nadof, tid, NT);
      } else {
        for (int i = tid; i < Jv * NMp; i += NT) {
          const int j = i / NMp, kk = i - j * NMp;
          XFr[i] = (j < J && kk < nm) ? p.t.XFt[(long long)kk * nadof + qb * A + j] : T(0);
        }
        for (int i = tid; i < Jv * NMp; i += NT) {
          const int j = i / NMp, kk = i - j * NMp;
          Xd[i] = (j < J && kk < nm) ? p.t.X[(long long)(qb * A + j) * nm + kk] : T(0);
        }
        for (int i = tid; i < Jv * Jp; i += NT) {
          const int j = i / Jp, j2 = i - j * Jp;
          SLr[i] = (j < J && j2 < J) ? p.SLD[((size_t)d * p.Jmax + j) * p.Jmax + j2] : T(0);
        }
      }
      stage_ad<T, DIM, A>(p, Ad, qb, J, tid, NT);
      // this thread's face word (axis, face node, unknown), if it polls one
      const int npoll = NF * HS * J;
      int pa = 0, pjn = 0, pj = 0;
      if (tid < npoll) {
        pa = tid / (HS * J);
        const int rem = tid - pa * HS * J;
        pjn = rem / J;
        pj = rem - pjn * J;
      }
      __syncthreads();
      stage_w<T, DIM, A>(p, Tin, Ad, Wl, lj_d, J, Jv, Ev, Evp, Eyl, Wp, n1, n2, tid, NT);
      __syncthreads();
      for (int ri = 0;; ++ri) {
        const int R = row_of(d, ri);
        if (R < 0) break;
        const int iy = R % g.ny, iz = R / g.ny;
        const int jy = n1 ? g.ny - 1 - iy : iy;
        const int jz = n2 ? g.nz - 1 - iz : iz;
        for (int k = 0; k < nx; ++k) {
          const long long c = c_next;
          const int slot = (int)(kc & 1);
          T* buf = bufs + (size_t)slot * Ev;
          T* phs = phss + (size_t)slot * S * NMp;
          const int mat = pmat;
          const T sig_s = psig;
          // ---- 1: the cell's data into shared memory; first look at the faces;
          //         the previous cell's moment update
#pragma unroll
          for (int u = 0; u < UM; ++u) {
            const int pe = tid + u * NT;
            if (pe < Ev) {
              rhs[pe] = pf[u];
              xold[pe] = px[u];
            }
          }
          if (c != last) {
#pragma unroll
            for (int u = 0; u < MM; ++u) {
              const int e = tid + u * NT;
              if (e < S * nm) {
                const int lk = slk[e];
                phs[(lk >> 16) * NMp + (lk & 0xffff)] = pm[u];
              }
            }
          }
          bool need = false;
          const unsigned long long* wp = nullptr;
          unsigned long long fw[W];
          if (tid < npoll) {
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
          if (pend) update_moments(last, slot ^ 1, c == last, d);
          __syncthreads();
          // ---- 2: the next cell of this block's sequence into registers;
          //         buf = X_d F Phi - S_dd^{L+D} x_old (four lanes per unknown)
          {
            int d2 = d, ri2 = ri, k2 = k + 1, sw2 = sw, R2 = R;
            bool more = true;
            if (k2 >= nx) {
              k2 = 0;
              ++ri2;
              R2 = row_of(d2, ri2);
              if (R2 < 0) {
                ri2 = 0;
                if (++d2 >= ndir) {
                  d2 = 0;
                  more = ++sw2 < p.sweeps;
                }
                if (more) R2 = row_of(d2, ri2);
              }
            }
            if (more) prefetch(d2, R2, k2);
            else c_next = -2;
            cp_async_commit_group();  // one group per cell, possibly empty
          }
          for (int base = 0; base < Ev; base += NQ) {
            // quads in (j, l) order: the S quads of one j share its row of
            // XFr (one 64-byte read serves them)
            const int pq = base + qd;
            const int pe = pq < Ev ? (pq & (S - 1)) * Jv + pq / S : Ev;
            const int lj = pe < Ev ? lj_d[pe] : -1;
            T a = T(0);
            if (lj >= 0) {
              const int l = lj >> 16, j = lj & 0xffff;
              const T* xr = XFr + j * NMp;
              const T* ph = phs + l * NMp;
              // two partial sums and an unrolled loop: the loads of several
              // chunks are in flight together
              T a1 = T(0);
#pragma unroll 4
              for (int ch = l4 * VW, it = 0; ch < NMp; ch += 4 * VW, ++it) {
                const T v = V16<T>::dot(xr + ch, ph + ch);
                if (it & 1) a1 += v;
                else a += v;
              }
              a += a1;
              if (!dense) {
                const T* sl = SLr + j * Jp;
                const T* xo = xold + l * Jv;
                for (int ch = l4 * VW; ch < Jv; ch += 4 * VW) a -= V16<T>::dot(sl + ch, xo + ch);
              }
            }
            a += __shfl_xor_sync(0xffffffffu, a, 1);
            a += __shfl_xor_sync(0xffffffffu, a, 2);
            if (pe < Ev && l4 == 0) buf[pe] = a;
          }
          // staged materials take the y/z inflow after the block solve:
          // rhs0 leaves it out, y0 = Tinv rhs0, then x = y0 + W yup
          // (rows on the inflow boundary have nothing to wait for)
          const bool late = mat < p.nmat_s && (jy > 0 || (DIM == 3 && jz > 0));
          auto wait_faces = [&]() {
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
            } else if (tid < npoll) {
              yup[(pa * HS + pjn) * Jv + pj] = T(0);  // a boundary face: no inflow here
            }
          };
          // the upwind rows' face words
          if (!late) wait_faces();
          __syncthreads();
          // ---- 3: rhs = f - upwind + sigma_s N buf (x only when late)
          for (int pe = tid; pe < Ev; pe += NT) {
            const int lj = lj_d[pe];
            if (lj < 0) continue;
            const int l = lj >> 16, j = lj & 0xffff;
            const int jq = j / A, m = j - jq * A, jb = jq * A;
            T val = rhs[pe];
#pragma unroll
            for (int xi = 0; xi < DIM; ++xi) {
              if (late && xi > 0) continue;
              const int own = xi == 0 ? n0 : (xi == 1 ? n1 : n2);
              const int jr = xi == 0 ? k : (xi == 1 ? jy : jz);
              if (jr == 0 || ((l >> xi) & 1) != own) continue;
              const T* up = xi == 0 ? xfc : yup + (size_t)(xi - 1) * HS * Jv;
              const T* An = Ad + ((size_t)jq * DIM + xi) * A * A + m * A;
              const int jp = fcompress(l, xi);
              T acc = T(0);
#pragma unroll
              for (int jn = 0; jn < HS; ++jn) {
                T sacc = T(0);
#pragma unroll
                for (int dd = 0; dd < A; ++dd) sacc += An[dd] * up[jn * Jv + jb + dd];
                acc += T(g.facemass[xi][jp][jn]) * sacc;
              }
              val -= (own ? T(1) : T(-1)) * acc;
            }
            T mix = T(0);
#pragma unroll
            for (int i = 0; i < S; ++i) mix += Ns[l * S + i] * buf[i * Jv + j];
            rhs[pe] = val + sig_s * mix;
          }
          cp_async_wait_prior();  // this cell's inverse (the next cell's may still fly)
          __syncthreads();
          // ---- 4: x_new = Tinv rhs (four lanes per row); outputs
          auto emit = [&](int pe, int lj, T a) {
            if (lj >= 0) {
              const int l = lj >> 16, j = lj & 0xffff;
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
          };
          for (int base = 0; base < Ev; base += NQ) {
            const int pe = base + qd;
            const int lj = pe < Ev ? lj_d[pe] : -1;
            T a = T(0);
            if (lj >= 0) {
              if (mat < p.nmat_s) {
                const T* row = Tin + ((size_t)mat * Ev + pe) * Evp;
                T a1 = T(0);
#pragma unroll 4
                for (int ch = l4 * VW, it = 0; ch < Ev; ch += 4 * VW, ++it) {
                  const T v = V16<T>::dot(row + ch, rhs + ch);
                  if (it & 1) a1 += v;
                  else a += v;
                }
                a += a1;
              } else if (p.gbuf > 0) {
                const int r = (lj >> 16) * J + (lj & 0xffff);
                const T* col = Tg + (size_t)(kc & 1) * p.gbuf + r;
                for (int cc = l4; cc < E; cc += 4) {
                  const int lc = cc / J;
                  a += col[(size_t)cc * p.Emax] * rhs[lc * Jv + (cc - lc * J)];
                }
              } else {
                const int r = (lj >> 16) * J + (lj & 0xffff);
                const T* col = p.TinvT + ((size_t)mat * ndir + d) * p.Emax * p.Emax + r;
                for (int cc = l4; cc < E; cc += 4) {
                  const int lc = cc / J;
                  a += __ldg(col + (size_t)cc * p.Emax) * rhs[lc * Jv + (cc - lc * J)];
                }
              }
            }
            a += __shfl_xor_sync(0xffffffffu, a, 1);
            a += __shfl_xor_sync(0xffffffffu, a, 2);
            if (pe < Ev && l4 == 0) {
              if (late) y0[pe] = a;
              else emit(pe, lj, a);
            }
          }
          if (late) {
            // ---- 5: the other rows' face values, then x = y0 + W yup
            wait_faces();
            __syncthreads();
            for (int base = 0; base < Ev; base += NQ) {
              const int pe = base + qd;
              const int lj = pe < Ev ? lj_d[pe] : -1;
              T a = T(0);
              if (lj >= 0 && NF > 0) {
                const T* wr = Wl + ((size_t)mat * Ev + pe) * Wp;
                for (int ch = l4 * VW; ch < Eyl; ch += 4 * VW) a += V16<T>::dot(wr + ch, yup + ch);
              }
              a += __shfl_xor_sync(0xffffffffu, a, 1);
              a += __shfl_xor_sync(0xffffffffu, a, 2);
              if (pe < Ev && l4 == 0) emit(pe, lj, y0[pe] + a);
            }
          }
          __syncthreads();
          last = c;
          pend = true;
          ++kc;
        }
      }
    }
  }
  if (pend) update_moments(last, (int)((kc - 1) & 1), false, 0);
  cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// Register form of the row-pipelined Gauss-Seidel: the dense form in FP32 on
// 2D Lin meshes with every material staged (at most two), at most 24
// unknowns per node and direction and at most 96 angular unknowns.  The
// per-cell work of the kernel above is a few short products with the
// direction's fixed matrices, so here each thread keeps its share of them in
// registers for the whole direction pass: M_d (warp w: rows j = w, w + 16;
// lane: columns 3 lane .. 3 lane + 2), each material's block inverse (warp w:
// rows 6 w .. 6 w + 5, the same columns) and its late-inflow table W (half
// warp h: rows 6 w + 3 h .. 6 w + 3 h + 2; columns 3 (lane mod 16) ..).  The
// vectors are read from shared memory by consecutive lanes (no bank
// conflicts), the partial sums reduced across the warp with the result
// spread over lane groups, and a cell takes three block barriers:
//   1  buf = M_d x_c, rhs0 = f - x-upwind + sigma_s N buf (N mixes the nodes
//      held by one warp: shuffles); the next cell's vectors start loading
//      into registers;
//   2  y0 = Tinv rhs0; the face words of the upwind row;
//   3  x = y0 + W yup, stores (psi, the x- and y-outflow faces), then the
//      next cell's vectors into shared memory (measured against a separate
//      staging phase: 45.3 against 47.8 ms per 10 sweeps on the 256^2 beam
//      workload; a three-cell cp.async ring was slower still).
// Schedule, face words, tags and waits are those of the kernel above.
constexpr int kFastThreads = 512;

// sum over the warp of v[0..7]; lane L receives the sum of v[(L >> 2) & 7]
// (the index halves at each of the first three exchange levels)
__device__ __forceinline__ float warp_sum8(const float (&v)[8], int lane) {
  const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
  float a[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    a[i] = (b4 ? v[i + 4] : v[i]) + __shfl_xor_sync(0xffffffffu, b4 ? v[i] : v[i + 4], 16);
  float c[2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
    c[i] = (b3 ? a[i + 2] : a[i]) + __shfl_xor_sync(0xffffffffu, b3 ? a[i] : a[i + 2], 8);
  float e = (b2 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, b2 ? c[0] : c[1], 4);
  e += __shfl_xor_sync(0xffffffffu, e, 2);
  e += __shfl_xor_sync(0xffffffffu, e, 1);
  return e;
}
// sum over a half warp of v[0..3]; lane L receives the sum of v[(L >> 2) & 3]
__device__ __forceinline__ float half_sum4(const float (&v)[4], int lane) {
  const bool b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
  float c[2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
    c[i] = (b3 ? v[i + 2] : v[i]) + __shfl_xor_sync(0xffffffffu, b3 ? v[i] : v[i + 2], 8);
  float e = (b2 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, b2 ? c[0] : c[1], 4);
  e += __shfl_xor_sync(0xffffffffu, e, 2);
  e += __shfl_xor_sync(0xffffffffu, e, 1);
  return e;
}

// the fast form applies: FP32 dense form, 2D Lin patches, every material
// staged (at most two), J <= 24 and nadof <= 96
__host__ __device__ inline bool rows_fast_applies(int dim, int a, int nadof, int Jmax, int nmat,
                                                  int nmat_s) {
  return dim == 2 && a == 3 && nadof <= 96 && Jmax <= 24 && nmat <= 2 && nmat_s == nmat;
}

template <int NMAT>
__global__ void __launch_bounds__(kFastThreads, 1) coarse_gs_rows_fast_kernel(RowsArgs<float> p) {
  using T = float;
  constexpr int DIM = 2, S = 4, HS = 2, A = 3;
  constexpr int W = FaceWords<T>::W;
  const Geom& g = p.g;
  const int nadof = g.nadof, nx = g.nx, ndir = p.ndir;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NT = blockDim.x;
  const int nb = gridDim.x, b = blockIdx.x;
  const RowsLayout<T> Ly(p.nmat_s, p.Jmax, nadof, S, DIM, A, ndir, 0, true);
  const int Jv = Ly.Jv, Ev = Ly.Ev, Evp = Ly.Evp, NMp = Ly.NMp, Eyl = Ly.Eyl, Wp = Ly.Wp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Tin = reinterpret_cast<T*>(smem_raw + Ly.o_Tin);    // [nmat_s][Ev][Evp]
  T* Md = reinterpret_cast<T*>(smem_raw + Ly.o_XFr);     // [Jv][NMp]
  T* Ns = reinterpret_cast<T*>(smem_raw + Ly.o_Ns);      // [S][S]
  T* Ad = reinterpret_cast<T*>(smem_raw + Ly.o_Ad);      // [patch][axis][A][A]
  int* slj = reinterpret_cast<int*>(smem_raw + Ly.o_lj); // [ndir][Ev] l<<16|j, -1 past J
  T* rhs = reinterpret_cast<T*>(smem_raw + Ly.o_rhs);    // [S][Jv] rhs0
  T* fb = reinterpret_cast<T*>(smem_raw + Ly.o_xold);    // [S][Jv] f of the direction block
  T* xc = reinterpret_cast<T*>(smem_raw + Ly.o_phs);     // [S][NMp] the cell's unknowns
  T* xfc = reinterpret_cast<T*>(smem_raw + Ly.o_xfc);    // [HS][Jv] x-outflow of the last cell
  T* yup = reinterpret_cast<T*>(smem_raw + Ly.o_yup);    // [HS][Jv] y inflow
  T* Wl = reinterpret_cast<T*>(smem_raw + Ly.o_W);       // [nmat_s][Ev][Wp]
  __shared__ int sdb[8], sde[8];
  if (tid < ndir) {
    sdb[tid] = p.dir_begin[tid];
    sde[tid] = p.dir_end[tid];
  }
  for (int i = tid; i < S * S; i += NT) Ns[i] = (T)g.Nmass[i];
  for (int i = tid; i < Eyl; i += NT) yup[i] = T(0);
  for (int i = tid; i < HS * Jv; i += NT) xfc[i] = T(0);
  for (int i = tid; i < ndir * Ev; i += NT) {
    const int d = i / Ev, pe = i - d * Ev;
    const int J = (p.dir_end[d] - p.dir_begin[d]) * A;
    const int l = pe / Jv, j = pe - l * Jv;
    slj[i] = j < J ? (l << 16) | j : -1;
  }
  const int* myrows = p.rows + (size_t)b * p.rpb;
  auto row_of = [&](int d, int ri) -> int {
    return ri < p.rpb ? myrows[(size_t)d * nb * p.rpb + ri] : -1;
  };
  const T fm00 = T(g.facemass[0][0][0]), fm01 = T(g.facemass[0][0][1]);
  const T fm10 = T(g.facemass[0][1][0]), fm11 = T(g.facemass[0][1][1]);
  __syncthreads();
  // prefetch registers: one value of x_c (threads < S nadof) or of f (the
  // next Ev threads), the material and sigma_s
  T xpf = T(0), fpf = T(0);
  int pmat = 0;
  T psig = T(0);
  long long c_next = -1;
  const int nxc = S * nadof;
  auto prefetch = [&](int d, int R, int k) {
    const int n0 = (d >> 1) & 1;
    const long long c = (n0 ? nx - 1 - k : k) + (long long)nx * R;
    c_next = c;
    if (tid < nxc) {
      xpf = __ldcg(p.psi + c * nxc + tid);
    } else if (tid < nxc + Ev) {
      const int e = tid - nxc, l = e / Jv, j = e - (e / Jv) * Jv;
      const int J = (sde[d] - sdb[d]) * A;
      fpf = j < J ? p.f[(c * S + l) * nadof + sdb[d] * A + j] : T(0);
    }
    pmat = p.cd.mat[c];
    psig = p.cd.sigma_s32[c];
  };
  // the cell whose vectors are in shared memory, and the prefetched one's
  // commit into it (x_c stays when the next cell is this one: its direction
  // block was updated in place)
  long long c_cur = -1;
  int mat_cur = 0;
  T sig_cur = T(0);
  auto commit = [&](bool same) {
    if (!same && tid < nxc) xc[(tid / nadof) * NMp + (tid - (tid / nadof) * nadof)] = xpf;
    if (tid >= nxc && tid < nxc + Ev) fb[tid - nxc] = fpf;
    c_cur = c_next;
    mat_cur = pmat;
    sig_cur = psig;
  };
  if (p.sweeps > 0) {
    prefetch(0, row_of(0, 0), 0);
    commit(false);
  }
  float Mr[2][3], Tr[NMAT][6][3], Wr[NMAT][3][3];
  const int h = lane >> 4;
  // face word of the upwind row: looked at once when the previous cell ends
  const unsigned long long* wp = nullptr;
  unsigned long long fw[W];
  bool looked = false;
  for (int sw = 0; sw < p.sweeps; ++sw) {
    const unsigned tag = p.tag0 + (unsigned)sw + 1u;
    for (int d = 0; d < ndir; ++d) {
      const int n0 = (d >> 1) & 1, n1 = d & 1;
      const int qb = sdb[d];
      const int J = (sde[d] - qb) * A;
      __syncthreads();  // the last direction's cells are done with the tables
      stage_tinv(p, Tin, d, J, Jv, Ev, Evp, tid, NT);
      stage_md(p, Md, d, qb * A, J, Jv, NMp, nadof, tid, NT);
      stage_ad<T, DIM, A>(p, Ad, qb, J, tid, NT);
      __syncthreads();
      stage_w<T, DIM, A>(p, Tin, Ad, Wl, slj + d * Ev, J, Jv, Ev, Evp, Eyl, Wp, n1, 0, tid, NT);
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          const int j = warp + 16 * r, k = 3 * lane + t;
          Mr[r][t] = (j < Jv && k < NMp) ? Md[j * NMp + k] : T(0);
        }
#pragma unroll
      for (int mt = 0; mt < NMAT; ++mt) {
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            const int e = 6 * warp + i, cc = 3 * lane + t;
            Tr[mt][i][t] = (mt < p.nmat_s && e < Ev && cc < Ev) ? Tin[((size_t)mt * Ev + e) * Evp + cc]
                                                                : T(0);
          }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            const int e = 6 * warp + 3 * h + i, cc = 3 * (lane & 15) + t;
            Wr[mt][i][t] = (mt < p.nmat_s && e < Ev && cc < Eyl) ? Wl[((size_t)mt * Ev + e) * Wp + cc]
                                                                 : T(0);
          }
      }
      // this thread's face word (face node, unknown), if it polls one
      const int npoll = HS * J;
      const int pjn = tid < npoll ? tid / J : 0, pj = tid < npoll ? tid - (tid / J) * J : 0;
      for (int ri = 0;; ++ri) {
        const int R = row_of(d, ri);
        if (R < 0) break;
        const int jy = n1 ? g.ny - 1 - R : R;
        for (int k = 0; k < nx; ++k) {
          const long long c = c_cur;
          const int mat = mat_cur;
          const T sig_s = sig_cur;
          // the next cell of this block's sequence: its vectors start loading
          // now and are committed when this cell ends
          int d2 = d, ri2 = ri, k2 = k + 1, sw2 = sw, R2 = R;
          bool more = true;
          if (k2 >= nx) {
            k2 = 0;
            ++ri2;
            R2 = row_of(d2, ri2);
            if (R2 < 0) {
              ri2 = 0;
              if (++d2 >= ndir) {
                d2 = 0;
                more = ++sw2 < p.sweeps;
              }
              if (more) R2 = row_of(d2, ri2);
            }
          }
          if (more) prefetch(d2, R2, k2);
          else c_next = -2;
          const bool need = tid < npoll && jy > 0;
          if (need && !looked) {
            const long long cn = c + (n1 ? (long long)nx : -(long long)nx);
            wp = p.faces + ((((size_t)0 * ndir + d) * g.C + cn) * HS * p.Jmax + (size_t)pjn * J + pj) * W;
            FaceWords<T>::load(wp, fw);
          }
          looked = false;
          // ---- 2: buf = M_d x_c; rhs0 = f - x-upwind + sigma_s N buf
          {
            float v[8];
            float xv[4][3];
#pragma unroll
            for (int l = 0; l < 4; ++l)
#pragma unroll
              for (int t = 0; t < 3; ++t) {
                const int kk = 3 * lane + t;
                xv[l][t] = kk < nadof ? xc[l * NMp + kk] : T(0);  // (padding unset)
              }
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
              for (int l = 0; l < 4; ++l)
                v[r * 4 + l] = Mr[r][0] * xv[l][0] + Mr[r][1] * xv[l][1] + Mr[r][2] * xv[l][2];
            const float tot = warp_sum8(v, lane);
            const int grp = (lane >> 2) & 7, r = grp >> 2, l = grp & 3;
            float bi[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) bi[i] = __shfl_sync(0xffffffffu, tot, ((r << 2) | i) << 2);
            const int j = warp + 16 * r;
            if ((lane & 3) == 0 && j < Jv) {
              T val = T(0);
              if (j < J) {
                const T mix = Ns[l * S + 0] * bi[0] + Ns[l * S + 1] * bi[1] + Ns[l * S + 2] * bi[2] +
                              Ns[l * S + 3] * bi[3];
                val = fb[l * Jv + j] + sig_s * mix;
                if (k > 0 && (l & 1) == n0) {
                  const int jq = j / A, m = j - jq * A, jp = l >> 1;
                  const T* An = Ad + ((size_t)jq * DIM + 0) * A * A + m * A;
                  const T* u0 = xfc + jq * A;
                  const T* u1 = xfc + Jv + jq * A;
                  const T s0 = An[0] * u0[0] + An[1] * u0[1] + An[2] * u0[2];
                  const T s1 = An[0] * u1[0] + An[1] * u1[1] + An[2] * u1[2];
                  const T acc = jp ? fm10 * s0 + fm11 * s1 : fm00 * s0 + fm01 * s1;
                  val -= (n0 ? T(1) : T(-1)) * acc;
                }
              }
              rhs[l * Jv + j] = val;
            }
          }
          __syncthreads();
          // ---- 3: y0 = Tinv rhs0; the upwind row's face values
          float y0;
          {
            float rv[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) rv[t] = 3 * lane + t < Ev ? rhs[3 * lane + t] : T(0);
            float v[8];
            v[6] = v[7] = 0.f;
            if (NMAT == 1 || mat == 0) {
#pragma unroll
              for (int i = 0; i < 6; ++i) v[i] = Tr[0][i][0] * rv[0] + Tr[0][i][1] * rv[1] + Tr[0][i][2] * rv[2];
            } else {
#pragma unroll
              for (int i = 0; i < 6; ++i)
                v[i] = Tr[NMAT - 1][i][0] * rv[0] + Tr[NMAT - 1][i][1] * rv[1] + Tr[NMAT - 1][i][2] * rv[2];
            }
            y0 = warp_sum8(v, lane);
          }
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
            yup[pjn * Jv + pj] = FaceWords<T>::value(fw);
          }
          __syncthreads();
          // ---- 4: x = y0 + W yup; outputs
          {
            float wy = 0.f;
            if (jy > 0) {
              float yv[3];
#pragma unroll
              for (int t = 0; t < 3; ++t) {
                const int cc = 3 * (lane & 15) + t;
                yv[t] = cc < Eyl ? yup[cc] : T(0);
              }
              float v[4];
              v[3] = 0.f;
              if (NMAT == 1 || mat == 0) {
#pragma unroll
                for (int i = 0; i < 3; ++i) v[i] = Wr[0][i][0] * yv[0] + Wr[0][i][1] * yv[1] + Wr[0][i][2] * yv[2];
              } else {
#pragma unroll
                for (int i = 0; i < 3; ++i)
                  v[i] = Wr[NMAT - 1][i][0] * yv[0] + Wr[NMAT - 1][i][1] * yv[1] + Wr[NMAT - 1][i][2] * yv[2];
              }
              wy = half_sum4(v, lane);
            }
            const int ip = (lane >> 2) & 3;
            const float y0v = __shfl_sync(0xffffffffu, y0, (4 * (3 * h + ip)) & 31);
            const int e = 6 * warp + 3 * h + ip;
            if ((lane & 3) == 0 && ip < 3 && e < Ev) {
              const int l = e / Jv, j = e - (e / Jv) * Jv;
              if (j < J) {
                const T x = y0v + wy;
                p.psi[(c * S + l) * nadof + qb * A + j] = x;
                if (c_next == c) xc[l * NMp + qb * A + j] = x;  // the next cell is this one
                if ((l & 1) != n0) xfc[(l >> 1) * Jv + j] = x;
                if (((l >> 1) & 1) != n1 && jy < g.ny - 1)
                  FaceWords<T>::put(p.faces + ((((size_t)0 * ndir + d) * g.C + c) * HS * p.Jmax +
                                               (size_t)(l & 1) * J + j) * W,
                                    x, tag);
              }
            }
          }
          // the next cell's vectors; a first look at its face word when it is
          // in this row
          if (more) {
            commit(c_next == c);
            if (d2 == d && R2 == R && tid < npoll && jy > 0) {
              const long long cn = c_next + (n1 ? (long long)nx : -(long long)nx);
              wp = p.faces + ((((size_t)0 * ndir + d) * g.C + cn) * HS * p.Jmax + (size_t)pjn * J + pj) * W;
              FaceWords<T>::load(wp, fw);
              looked = true;
            }
          }
          __syncthreads();
        }
      }
    }
  }
}

template <class T, int DIM, int A, class F>
auto with_rows_kernel(int shape, F f) {
  if (shape == 0) return f(coarse_gs_rows_kernel<T, DIM, A, 1, 1>);
  if (shape == 1) return f(coarse_gs_rows_kernel<T, DIM, A, 2, 2>);
  return f(coarse_gs_rows_kernel<T, DIM, A, 2, 8>);
}

template <class T, int DIM, int A>
cudaError_t rows_launch(const RowsArgs<T>& a, int shape, int nblocks, int threads, size_t smem,
                        cudaStream_t st) {
  return with_rows_kernel<T, DIM, A>(shape, [&](auto kern) {
    cudaError_t e = allow_max_smem(kern);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a};
    return cudaLaunchCooperativeKernel((void*)kern, dim3(nblocks), dim3(threads), args, smem, st);
  });
}

template <class T, int DIM, int A>
int rows_max_blocks(int shape, int threads, size_t smem) {
  return with_rows_kernel<T, DIM, A>(shape, [&](auto kern) {
    if (allow_max_smem(kern) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    int per_sm = 0, dev = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * nsm;
  });
}

}  // namespace

template <class T>
int coarse_gs_rows_plan(const Geom& g, int ndir, int nmat, int Jmax, int nmom, bool dense,
                        int* nmat_s, int* threads, size_t* smem, int* gbuf) {
  if (g.a != 1 && g.a != 3) return 0;
  const int S = g.s;
  if (dense) nmom = g.nadof;  // the cell vector x_c in the moments' place
  // four lanes per padded unknown and per moment, within one block
  const RowsLayout<T> l0(0, Jmax, nmom, S, g.dim, g.a, ndir, 0, dense);
  int nt = 4 * std::max(l0.Ev, S * nmom);
  nt = std::max(128, std::min(kRowsMaxThreads, (nt + 31) / 32 * 32));
  if (l0.Ev > kRowsMaxU * nt || S * nmom > kRowsMaxM * nt || (g.dim - 1) * (S / 2) * Jmax > nt ||
      g.nx < 1)
    return 0;
  // materials whose inverses are staged per direction; the others are
  // prefetched cell by cell into two buffers (when those fit)
  const int Emax = S * Jmax;
  int gb = 0;
  auto bytes_for = [&](int ns) {
    return RowsLayout<T>(ns, Jmax, nmom, S, g.dim, g.a, ndir, ns < nmat ? gb : 0, dense).bytes;
  };
  gb = Emax * Emax;
  if (RowsLayout<T>(0, Jmax, nmom, S, g.dim, g.a, ndir, gb, dense).bytes > 200 * 1024) gb = 0;
  int ns = nmat;
  while (ns > 0 && bytes_for(ns) > 200 * 1024) --ns;
  const size_t bytes = bytes_for(ns);
  if (bytes > 200 * 1024) return 0;
  *gbuf = ns < nmat ? gb : 0;
  const int shape = rows_shape(l0.Ev, S * nmom, nt);
  int nb;
  if constexpr (sizeof(T) == 4) {
    if (dense && rows_fast_applies(g.dim, g.a, g.nadof, Jmax, nmat, ns)) {
      // the register form: 512 threads, one launch shape per material count
      int per_sm = 0;
      auto kern = nmat == 1 ? coarse_gs_rows_fast_kernel<1> : coarse_gs_rows_fast_kernel<2>;
      if (allow_max_smem(kern) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFastThreads, bytes) !=
              cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
      }
      int dev = 0, nsm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      *nmat_s = ns;
      *threads = kFastThreads;
      *smem = bytes;
      return std::min(per_sm * nsm, g.ny * g.nz);
    }
  }
  if (g.dim == 2)
    nb = g.a == 3 ? rows_max_blocks<T, 2, 3>(shape, nt, bytes)
                  : rows_max_blocks<T, 2, 1>(shape, nt, bytes);
  else
    nb = g.a == 3 ? rows_max_blocks<T, 3, 3>(shape, nt, bytes)
                  : rows_max_blocks<T, 3, 1>(shape, nt, bytes);
  nb = std::min(nb, g.ny * g.nz);
  *nmat_s = ns;
  *threads = nt;
  *smem = bytes;
  return nb;
}

template <class T>
int launch_coarse_gs_rows(const Geom& g, const LevelDev<T>& t, const CellData& cd, int ndir,
                          const int* dir_begin, const int* dir_end, int sweeps, const T* f,
                          T* phi, T* mom, const T* TinvT, const T* SLD, const T* Sf, int Emax,
                          int Jmax, int nmat, int nmat_s, int gbuf, int threads, size_t smem,
                          const int* rows, int nblocks, int rpb, unsigned long long* faces,
                          unsigned tag0, int* err, cudaStream_t st) {
  const int dense = Sf != nullptr ? 1 : 0;
  RowsArgs<T> a{g, t, cd, ndir, dir_begin, dir_end, sweeps, f, phi, mom, TinvT, SLD, Sf, dense,
                Emax, Jmax, nmat, nmat_s, gbuf, rows, rpb, faces, tag0, err};
  const int nm = dense ? g.nadof : t.nmom;
  const RowsLayout<T> l0(0, Jmax, nm, g.s, g.dim, g.a, ndir, 0, dense != 0);
  const int shape = rows_shape(l0.Ev, g.s * nm, threads);
  cudaError_t e;
  bool fast = false;
  if constexpr (sizeof(T) == 4) {
    fast = dense && threads == kFastThreads && rows_fast_applies(g.dim, g.a, g.nadof, Jmax, nmat,
                                                                 nmat_s);
    if (fast) {
      auto kern = nmat == 1 ? coarse_gs_rows_fast_kernel<1> : coarse_gs_rows_fast_kernel<2>;
      e = allow_max_smem(kern);
      if (e == cudaSuccess) {
        void* args[] = {(void*)&a};
        e = cudaLaunchCooperativeKernel((void*)kern, dim3(nblocks), dim3(threads), args, smem, st);
      }
    }
  }
  if (fast) {
  } else if (g.dim == 2)
    e = g.a == 3 ? rows_launch<T, 2, 3>(a, shape, nblocks, threads, smem, st)
                 : rows_launch<T, 2, 1>(a, shape, nblocks, threads, smem, st);
  else
    e = g.a == 3 ? rows_launch<T, 3, 3>(a, shape, nblocks, threads, smem, st)
                 : rows_launch<T, 3, 1>(a, shape, nblocks, threads, smem, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  note_launch();
  return 0;
}

bool coarse_gs_rows_fast(const Geom& g, int Jmax, int nmat, int nmat_s, int threads) {
  return threads == kFastThreads && rows_fast_applies(g.dim, g.a, g.nadof, Jmax, nmat, nmat_s);
}

template int coarse_gs_rows_plan<float>(const Geom&, int, int, int, int, bool, int*, int*, size_t*,
                                        int*);
template int coarse_gs_rows_plan<double>(const Geom&, int, int, int, int, bool, int*, int*,
                                         size_t*, int*);
template int launch_coarse_gs_rows<float>(const Geom&, const LevelDev<float>&, const CellData&, int,
                                          const int*, const int*, int, const float*, float*,
                                          float*, const float*, const float*, const float*, int,
                                          int, int, int, int, int, size_t, const int*, int, int,
                                          unsigned long long*, unsigned, int*, cudaStream_t);
template int launch_coarse_gs_rows<double>(const Geom&, const LevelDev<double>&, const CellData&,
                                           int, const int*, const int*, int, const double*,
                                           double*, double*, const double*, const double*,
                                           const double*, int, int, int, int, int, int, size_t,
                                           const int*, int, int, unsigned long long*, unsigned,
                                           int*, cudaStream_t);

}  // namespace amgt
