// Host-side FP64 construction of the discretisation tables (angular patch
// hierarchy, bases, patch quadrature, angular matrices, spherical harmonics,
// Q1 spatial matrices, per-patch block matrices and their inverses).
// Everything here runs once per problem set-up; nothing is on the hot path.
#pragma once
#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace amgt {

struct Patch {
  double v[3][3];            // unit-vector vertices
  int octant = 0;
  int level = 0;
  std::vector<uint8_t> path; // octant, then child indices
};

// A mesh of patches with the basis and per-patch angular tables
// (Sec. 2.2-2.3): w = int Psi, M = int Psi Psi, A^xi = int Omega_xi Psi Psi,
// Aw = int Omega_xi Psi.
struct AngMesh {
  int basis = 1;  // 0 Const, 1 Lin
  int a = 3;
  int P = 0;
  std::vector<Patch> patch;
  std::vector<double> w;   // [P][a]
  std::vector<double> M;   // [P][a][a]
  std::vector<double> A;   // [P][3][a][a]
  std::vector<double> Aw;  // [P][3][a]
  int nadof() const { return P * a; }
};

std::vector<std::vector<uint8_t>> uniform_paths(int level);
std::vector<std::vector<uint8_t>> aniso_paths(int lmax, const double axis[3]);
std::vector<std::vector<uint8_t>> coarsen_paths(const std::vector<std::vector<uint8_t>>& paths,
                                                int level);
int max_level(const std::vector<std::vector<uint8_t>>& paths);
AngMesh build_mesh(const std::vector<std::vector<uint8_t>>& paths, int basis);

// basis values Psi_d(omega) on patch p (omega inside the patch), out[a]
void basis_values(const AngMesh& m, int p, const double om[3], double* out);

// patch quadrature: nodes (unit vectors) and weights
void patch_quadrature(const Patch& p, int order, std::vector<double>& nodes,
                      std::vector<double>& weights);
int quadrature_order(int level, int N);

// real orthonormal harmonics of degree <= N at omega, out[(N+1)^2]
void real_harmonics(int N, const double om[3], double* out);

// X[P*a][(N+1)^2] = int Psi Y (Sec. 4.2)
std::vector<double> x_table(const AngMesh& m, int N);

// Pencil-beam inflow weights at the beam direction om (Sec. 5.4): the Dirac
// mass goes to the patches whose closed spherical triangle holds om, each
// with the fraction of an infinitesimal cap around om that lies in it (1
// inside, 1/2 on an edge, the interior angle / 2 pi at a vertex); writes
// out[q a + m] = fac share_q Psi_[q]m(om) for those patches only and returns
// the sum of the shares (1 when the mesh covers om).
double beam_weights(const AngMesh& m, const double om[3], double fac, double* out);

// prolongation between nested meshes: parent[f], Pblk[f][a][a] with
// Pblk[f][k][d] = Psi_{parent,d}(vertex k of f); child ranges per coarse patch
struct Transfer {
  std::vector<int> parent;       // [Pf]
  std::vector<double> blk;       // [Pf][a][a]
  std::vector<int> child_begin;  // [Pc]
  std::vector<int> child_end;    // [Pc]
};
Transfer build_transfer(const AngMesh& fine, const AngMesh& coarse);

// Q1 element matrices on a box cell with widths h (closed forms)
struct Q1 {
  int dim = 2, s = 4;
  double h[3] = {1, 1, 1};
  std::vector<double> N;      // [s][s]
  std::vector<double> V;      // [dim][s][s]
  std::vector<double> Fown;   // [2dim][s][s]
  std::vector<double> Fnb;    // [2dim][s][s]
  std::vector<double> mu;     // [s]
  std::vector<double> mf;     // [2dim][s]
  std::vector<double> facemass;  // [dim][s/2][s/2] own face node j' x neighbour face node j
};
Q1 build_q1(int dim, const double h[3]);
// node index with bit `axis` set to `bit` and the other bits taken from j
inline int face_node(int j, int axis, int bit) {
  int lo = j & ((1 << axis) - 1);
  int hi = (j >> axis) << (axis + 1);
  return lo | (bit << axis) | hi;
}

// dense inverse by Gaussian elimination with partial pivoting; false if singular
bool invert(int n, const double* A, double* Ainv);

}  // namespace amgt
