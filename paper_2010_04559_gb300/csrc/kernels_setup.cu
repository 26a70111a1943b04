// Set-up tables on the GPU: the block inverses of the sweep (Sec. 3), of the
// coarse Gauss-Seidel's block solves with self-scatter (Sec. 4.2) and of its
// direction-blocked form, one per material (distinct sigma_t, sigma_s, moment
// shape) and patch or sweep direction.  With a different sigma_t in every
// cell these are millions of small matrices; each thread block assembles one
// in shared memory and inverts it in place by Gauss-Jordan elimination with
// partial pivoting (row interchanges recorded, undone as column interchanges
// at the end), the same algorithm as the host's invert().
#include <cstdint>

#include "kernels.cuh"

namespace amgt {

namespace {

constexpr int kInvThreads = 256;

// One matrix per block.  kind 0: K0_q + st B_q (n = s a); kind 1: the same
// minus ss kron(N, S_qq) (coarse Gauss-Seidel block with self-scatter); kind
// 2: the direction-blocked matrix of direction d over e = l J + j:
// [p == q] (K0 + st B)_{(l,m),(i,dd)} - ss N[l][i] SLD[d][j][j2].
struct InvArgs {
  int kind, n, s, a, P, ndir, Jmax, Emax;
  const double* K0;      // [P][sa][sa]
  const double* B;       // [P][sa][sa]
  const double* Sqq;     // [nf][P][a][a]
  const double* SLD;     // [ndir][Jmax][Jmax]
  const int* dir_begin;  // [ndir]
  const int* dir_end;
  const double* mat_st;  // [nmat]
  const double* mat_ss;
  const int* mat_f;      // [nmat] moment shape (null: 0)
  double* out;           // kinds 0/1: [nmat][P][n][n]; kind 2: [nmat][ndir][Emax][Emax] transposed
  int* singular;
};

__global__ void __launch_bounds__(kInvThreads) invert_blocks_kernel(Geom g, InvArgs p) {
  extern __shared__ double A[];  // [n][n] (n = the matrix size of this block)
  __shared__ int perm_s[512];
  __shared__ int piv_s;
  __shared__ double red_v[kInvThreads / 32];
  __shared__ int red_i[kInvThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long blk = blockIdx.x;
  int mt, q = 0, d = 0, n = p.n, qb = 0, J = 0;
  if (p.kind == 2) {
    mt = (int)(blk / p.ndir);
    d = (int)(blk - (long long)mt * p.ndir);
    qb = p.dir_begin[d];
    J = (p.dir_end[d] - qb) * p.a;
    n = p.s * J;
  } else {
    mt = (int)(blk / p.P);
    q = (int)(blk - (long long)mt * p.P);
  }
  const int sa = p.s * p.a;
  const double st = p.mat_st[mt], ss = p.mat_ss[mt];
  // assemble
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    double v;
    if (p.kind != 2) {
      const size_t o = (size_t)q * sa * sa + (size_t)r * sa + c;
      v = p.K0[o] + st * p.B[o];
      if (p.kind == 1) {
        const int l = r / p.a, m = r - l * p.a, i = c / p.a, dd = c - i * p.a;
        const int sh = p.mat_f ? p.mat_f[mt] : 0;
        v -= ss * g.Nmass[l * p.s + i] *
             p.Sqq[(((size_t)sh * p.P + q) * p.a + m) * p.a + dd];
      }
    } else {
      const int l = r / J, j = r - l * J, i = c / J, j2 = c - i * J;
      const int qq = j / p.a, m = j - qq * p.a, pp = j2 / p.a, dd = j2 - pp * p.a;
      v = 0.0;
      if (pp == qq) {
        const size_t o = (size_t)(qb + qq) * sa * sa + (size_t)(l * p.a + m) * sa + i * p.a + dd;
        v = p.K0[o] + st * p.B[o];
      }
      v -= ss * g.Nmass[l * p.s + i] * p.SLD[((size_t)d * p.Jmax + j) * p.Jmax + j2];
    }
    A[e] = v;
  }
  __syncthreads();
  bool bad = false;
  for (int k = 0; k < n; ++k) {
    // pivot: the largest |A[i][k]|, i >= k (lowest index on ties)
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < n; i += blockDim.x) {
      const double v = fabs(A[i * n + k]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      red_v[warp] = best;
      red_i[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double b = red_v[0];
      int ib = red_i[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (red_v[w] > b || (red_v[w] == b && red_i[w] < ib)) {
          b = red_v[w];
          ib = red_i[w];
        }
      piv_s = ib;
      perm_s[k] = ib;
    }
    __syncthreads();
    const int pr = piv_s;
    if (pr != k)
      for (int c = tid; c < n; c += blockDim.x) {
        const double t = A[k * n + c];
        A[k * n + c] = A[pr * n + c];
        A[pr * n + c] = t;
      }
    __syncthreads();
    const double pv = A[k * n + k];
    if (pv == 0.0) {
      bad = true;
      break;
    }
    const double inv = 1.0 / pv;
    __syncthreads();
    // row k: A[k][c] /= pv, with A[k][k] := 1 / pv
    for (int c = tid; c < n; c += blockDim.x) A[k * n + c] = (c == k ? 1.0 : A[k * n + c]) * inv;
    __syncthreads();
    // other rows: A[r][c] -= A[r][k] A[k][c], with A[r][k] := -A[r][k] / pv
    for (int e = tid; e < n * n; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      if (r == k || c == k) continue;
      A[e] -= A[r * n + k] * A[k * n + c];
    }
    __syncthreads();
    for (int r = tid; r < n; r += blockDim.x)
      if (r != k) A[r * n + k] = -A[r * n + k] * inv;
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) atomicExch(p.singular, 1);
    return;
  }
  // undo the row interchanges as column interchanges, last first
  for (int k = n - 1; k >= 0; --k) {
    const int pr = perm_s[k];
    if (pr != k)
      for (int r = tid; r < n; r += blockDim.x) {
        const double t = A[r * n + k];
        A[r * n + k] = A[r * n + pr];
        A[r * n + pr] = t;
      }
    __syncthreads();
  }
  if (p.kind != 2) {
    double* o = p.out + (size_t)blk * n * n;
    for (int e = tid; e < n * n; e += blockDim.x) o[e] = A[e];
  } else {
    double* o = p.out + ((size_t)mt * p.ndir + d) * p.Emax * p.Emax;
    // transposed, zero-padded to Emax
    for (int e = tid; e < p.Emax * p.Emax; e += blockDim.x) {
      const int cc = e / p.Emax, r = e - cc * p.Emax;
      o[e] = (r < n && cc < n) ? A[r * n + cc] : 0.0;
    }
  }
}

}  // namespace

int invert_blocks_max() { return 160; }

cudaError_t launch_invert_blocks(const Geom& g, int kind, int nmat, int P, int s, int a,
                                 const double* K0, const double* B, const double* Sqq,
                                 const double* SLD, int ndir, const int* dir_begin,
                                 const int* dir_end, int Jmax, int Emax, const double* mat_st,
                                 const double* mat_ss, const int* mat_f, double* out,
                                 int* singular, cudaStream_t st) {
  InvArgs p{kind, s * a, s, a, P, ndir, Jmax, Emax, K0, B, Sqq, SLD, dir_begin, dir_end,
            mat_st, mat_ss, mat_f, out, singular};
  const int nmax = kind == 2 ? Emax : s * a;
  if (nmax > invert_blocks_max() || nmax < 1) return cudaErrorInvalidValue;
  const size_t smem = (size_t)nmax * nmax * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(invert_blocks_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(invert_blocks_max() * invert_blocks_max() * 8));
  if (e != cudaSuccess) return e;
  const long long nblk = (long long)nmat * (kind == 2 ? ndir : P);
  const int threads = nmax <= 24 ? 64 : kInvThreads;
  note_launch();
  invert_blocks_kernel<<<(unsigned)nblk, threads, smem, st>>>(g, p);
  return cudaGetLastError();
}

}  // namespace amgt
