// Test-only C entry points over the library's host set-up code
// (paper_2010_04559_gb300/csrc/setup.cpp), compiled with it into a small
// shared library by tests/test_setup_tables_host.py so that the set-up
// tables can be compared with the oracle's on the CPU.  Not part of libamgt.
#include <cstring>
#include <vector>

#include "setup.hpp"

using namespace amgt;

namespace {
std::vector<std::vector<uint8_t>> mesh_paths(int level, int aniso, const double* axis) {
  return aniso ? aniso_paths(level, axis) : uniform_paths(level);
}
}  // namespace

extern "C" {

// Patches of the mesh (uniform of `level`, or band-refined about `axis` to
// lmax = level when aniso); paths[P][8] (octant then children, 255 = none).
int shim_paths(int level, int aniso, const double* axis, unsigned char* paths, int cap) {
  const auto ps = mesh_paths(level, aniso, axis);
  if (paths)
    for (size_t p = 0; p < ps.size() && (int)p < cap; ++p)
      for (int k = 0; k < 8; ++k) paths[p * 8 + k] = k < (int)ps[p].size() ? ps[p][k] : 255;
  return (int)ps.size();
}

// Angular tables w [P][a], M [P][a][a], A [P][3][a][a], Aw [P][3][a].
int shim_mesh(int level, int aniso, const double* axis, int basis, double* w, double* M,
              double* A, double* Aw) {
  const AngMesh m = build_mesh(mesh_paths(level, aniso, axis), basis);
  std::memcpy(w, m.w.data(), m.w.size() * sizeof(double));
  std::memcpy(M, m.M.data(), m.M.size() * sizeof(double));
  std::memcpy(A, m.A.data(), m.A.size() * sizeof(double));
  std::memcpy(Aw, m.Aw.data(), m.Aw.size() * sizeof(double));
  return m.P;
}

// X [P a][(N+1)^2] = int Psi Y.
void shim_xtable(int level, int aniso, const double* axis, int basis, int N, double* X) {
  const AngMesh m = build_mesh(mesh_paths(level, aniso, axis), basis);
  const std::vector<double> x = x_table(m, N);
  std::memcpy(X, x.data(), x.size() * sizeof(double));
}

// Dense prolongation [nadof_fine][nadof_coarse] from the mesh (as above)
// to the same mesh coarsened to `coarse_level`.
void shim_prolongation(int level, int aniso, const double* axis, int basis, int coarse_level,
                       double* P) {
  const auto fp = mesh_paths(level, aniso, axis);
  const AngMesh fine = build_mesh(fp, basis);
  const AngMesh coarse = build_mesh(coarsen_paths(fp, coarse_level), basis);
  const Transfer t = build_transfer(fine, coarse);
  const int a = fine.a, nc = coarse.nadof();
  std::memset(P, 0, sizeof(double) * (size_t)fine.nadof() * nc);
  for (int f = 0; f < fine.P; ++f)
    for (int k = 0; k < a; ++k)
      for (int d = 0; d < a; ++d)
        P[(size_t)(f * a + k) * nc + t.parent[f] * a + d] = t.blk[(f * a + k) * a + d];
}

// Q1 element matrices: N [s][s], V [dim][s][s], Fown, Fnb [2dim][s][s],
// mu [s], mf [2dim][s].
void shim_q1(int dim, const double* h, double* N, double* V, double* Fown, double* Fnb,
             double* mu, double* mf) {
  const Q1 q = build_q1(dim, h);
  std::memcpy(N, q.N.data(), q.N.size() * sizeof(double));
  std::memcpy(V, q.V.data(), q.V.size() * sizeof(double));
  std::memcpy(Fown, q.Fown.data(), q.Fown.size() * sizeof(double));
  std::memcpy(Fnb, q.Fnb.data(), q.Fnb.size() * sizeof(double));
  std::memcpy(mu, q.mu.data(), q.mu.size() * sizeof(double));
  std::memcpy(mf, q.mf.data(), q.mf.size() * sizeof(double));
}

int shim_invert(int n, const double* A, double* Ainv) { return invert(n, A, Ainv) ? 1 : 0; }

}  // extern "C"

extern "C" {

// Pencil-beam weights at direction om (fac = 1): out [P a] (zero outside the
// patches holding om); returns the sum of the shares.
double shim_beam(int level, int aniso, const double* axis, int basis, const double* om,
                 double* out) {
  const AngMesh m = build_mesh(mesh_paths(level, aniso, axis), basis);
  std::memset(out, 0, sizeof(double) * (size_t)m.nadof());
  return beam_weights(m, om, 1.0, out);
}

}  // extern "C"

extern "C" {

// Q1 face mass on the faces normal to each axis: facemass [dim][s/2][s/2].
void shim_q1_facemass(int dim, const double* h, double* out) {
  const Q1 q = build_q1(dim, h);
  std::memcpy(out, q.facemass.data(), q.facemass.size() * sizeof(double));
}

}  // extern "C"
