// Host FP64 set-up of the space-angle DG tables.
//
// Angular mesh (Sec. 2.1): octants o = 4bx + 2by + bz split recursively into
// four daughters by the great-circle edge midpoints normalize(a + b).
// Lin basis (Sec. 2.2): barycentric coordinates, in the flat triangle of the
// vertices projected onto the octahedron, of the central projection
// Omega / |Omega|_1.  Integrals over a patch (Sec. 2.3, Sec. 4.2) use the same
// central map, dOmega = |x|^-3 dA / sqrt(3), and a collapsed Gauss-Legendre
// product rule (collapse at the third vertex).  Spherical harmonics are real
// orthonormal with polar axis e_x; only their degree-n sums enter S, which by
// the addition theorem do not depend on that choice.
#include "setup.hpp"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <stdexcept>
#include <thread>
#include <vector>

namespace amgt {

namespace {

void unit(double* v) {
  double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  v[0] /= n; v[1] /= n; v[2] /= n;
}

void octant_verts(int o, double v[3][3]) {
  std::memset(v, 0, sizeof(double) * 9);
  v[0][0] = ((o >> 2) & 1) ? -1.0 : 1.0;
  v[1][1] = ((o >> 1) & 1) ? -1.0 : 1.0;
  v[2][2] = (o & 1) ? -1.0 : 1.0;
}

void child_verts(const double v[3][3], int c, double out[3][3]) {
  double ab[3], bc[3], ca[3];
  for (int e = 0; e < 3; ++e) {
    ab[e] = v[0][e] + v[1][e];
    bc[e] = v[1][e] + v[2][e];
    ca[e] = v[2][e] + v[0][e];
  }
  unit(ab); unit(bc); unit(ca);
  const double* pick[4][3] = {{v[0], ab, ca}, {ab, v[1], bc}, {ca, bc, v[2]}, {ab, bc, ca}};
  for (int k = 0; k < 3; ++k)
    for (int e = 0; e < 3; ++e) out[k][e] = pick[c][k][e];
}

void path_verts(const std::vector<uint8_t>& path, double v[3][3]) {
  octant_verts(path[0], v);
  for (size_t i = 1; i < path.size(); ++i) {
    double t[3][3];
    child_verts(v, path[i], t);
    std::memcpy(v, t, sizeof(t));
  }
}

// Gauss-Legendre nodes/weights on [0,1] by Newton iteration on P_n
void gauss01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_n(t), p0 = P_{n-1}(t)
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
    }
    x[i] = 0.5 * (1.0 - t);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);  // = 0.5 * 2/((1-t^2) P_n'^2)
  }
}

double band_target(const double v[3][3], const double axis[3], int lmax) {
  double m = -2.0;
  for (int k = 0; k < 3; ++k)
    m = std::max(m, v[k][0] * axis[0] + v[k][1] * axis[1] + v[k][2] * axis[2]);
  int t;
  if (m > 0.97) t = lmax;
  else if (m > 0.9) t = lmax - 1;
  else if (m > 0.8) t = lmax - 2;
  else if (m > 0.6) t = lmax - 3;
  else t = lmax - 4;
  return t < 0 ? 0 : t;
}

}  // namespace

std::vector<std::vector<uint8_t>> uniform_paths(int level) {
  std::vector<std::vector<uint8_t>> out;
  std::function<void(std::vector<uint8_t>&)> rec = [&](std::vector<uint8_t>& p) {
    if ((int)p.size() - 1 == level) {
      out.push_back(p);
      return;
    }
    for (int c = 0; c < 4; ++c) {
      p.push_back((uint8_t)c);
      rec(p);
      p.pop_back();
    }
  };
  for (int o = 0; o < 8; ++o) {
    std::vector<uint8_t> p{(uint8_t)o};
    rec(p);
  }
  return out;
}

std::vector<std::vector<uint8_t>> aniso_paths(int lmax, const double axis_in[3]) {
  double axis[3] = {axis_in[0], axis_in[1], axis_in[2]};
  unit(axis);
  std::vector<std::vector<uint8_t>> out;
  std::function<void(std::vector<uint8_t>&, const double (*)[3])> rec =
      [&](std::vector<uint8_t>& p, const double (*v)[3]) {
        int lev = (int)p.size() - 1;
        if (lev < band_target(v, axis, lmax)) {
          for (int c = 0; c < 4; ++c) {
            double cv[3][3];
            child_verts(v, c, cv);
            p.push_back((uint8_t)c);
            rec(p, cv);
            p.pop_back();
          }
        } else {
          out.push_back(p);
        }
      };
  for (int o = 0; o < 8; ++o) {
    double v[3][3];
    octant_verts(o, v);
    std::vector<uint8_t> p{(uint8_t)o};
    rec(p, v);
  }
  return out;
}

std::vector<std::vector<uint8_t>> coarsen_paths(const std::vector<std::vector<uint8_t>>& paths,
                                                int level) {
  std::vector<std::vector<uint8_t>> out;
  for (const auto& p : paths) {
    std::vector<uint8_t> q(p.begin(), p.begin() + std::min<size_t>(p.size(), level + 1));
    if (out.empty() || out.back() != q) out.push_back(q);
  }
  return out;
}

int max_level(const std::vector<std::vector<uint8_t>>& paths) {
  int m = 0;
  for (const auto& p : paths) m = std::max(m, (int)p.size() - 1);
  return m;
}

int quadrature_order(int level, int N) {
  return 20 + (int)std::ceil(1.75 * N / (double)(1 << level));
}

void patch_quadrature(const Patch& p, int order, std::vector<double>& nodes,
                      std::vector<double>& weights) {
  std::vector<double> t, wt;
  gauss01(order, t, wt);
  double u[3][3];
  for (int k = 0; k < 3; ++k) {
    double l1 = std::fabs(p.v[k][0]) + std::fabs(p.v[k][1]) + std::fabs(p.v[k][2]);
    for (int e = 0; e < 3; ++e) u[k][e] = p.v[k][e] / l1;
  }
  // x = u2 + xi * ((u0 - u2) + eta * (u1 - u0)), Jacobian xi * |e1 x e2|
  double e1[3], e2[3];
  for (int e = 0; e < 3; ++e) {
    e1[e] = u[0][e] - u[2][e];
    e2[e] = u[1][e] - u[0][e];
  }
  double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                  e1[0] * e2[1] - e1[1] * e2[0]};
  double twoA = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  const double h = 1.0 / std::sqrt(3.0);
  nodes.resize(3 * order * order);
  weights.resize(order * order);
  int k = 0;
  for (int i = 0; i < order; ++i)
    for (int j = 0; j < order; ++j, ++k) {
      double xi = t[i], eta = t[j];
      double x[3];
      for (int e = 0; e < 3; ++e) x[e] = u[2][e] + xi * (e1[e] + eta * e2[e]);
      double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
      for (int e = 0; e < 3; ++e) nodes[3 * k + e] = x[e] / r;
      weights[k] = wt[i] * wt[j] * xi * twoA * h / (r * r * r);
    }
}

void basis_values(const AngMesh& m, int p, const double om[3], double* out) {
  if (m.basis == 0) {
    out[0] = 1.0;
    return;
  }
  const Patch& P = m.patch[p];
  // columns u_k = v_k / |v_k|_1; solve U lam = om / (s . om) by Cramer's rule
  double U[3][3];
  for (int k = 0; k < 3; ++k) {
    double l1 = std::fabs(P.v[k][0]) + std::fabs(P.v[k][1]) + std::fabs(P.v[k][2]);
    for (int e = 0; e < 3; ++e) U[e][k] = P.v[k][e] / l1;
  }
  double s[3] = {((P.octant >> 2) & 1) ? -1.0 : 1.0, ((P.octant >> 1) & 1) ? -1.0 : 1.0,
                 (P.octant & 1) ? -1.0 : 1.0};
  double sd = s[0] * om[0] + s[1] * om[1] + s[2] * om[2];
  double x[3] = {om[0] / sd, om[1] / sd, om[2] / sd};
  auto det3 = [](const double M[3][3]) {
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
           M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
           M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
  };
  double D = det3(U);
  for (int k = 0; k < 3; ++k) {
    double Mk[3][3];
    std::memcpy(Mk, U, sizeof(U));
    for (int e = 0; e < 3; ++e) Mk[e][k] = x[e];
    out[k] = det3(Mk) / D;
  }
}

AngMesh build_mesh(const std::vector<std::vector<uint8_t>>& paths, int basis) {
  AngMesh m;
  m.basis = basis;
  m.a = basis == 0 ? 1 : 3;
  m.P = (int)paths.size();
  m.patch.resize(m.P);
  for (int p = 0; p < m.P; ++p) {
    Patch& P = m.patch[p];
    P.path = paths[p];
    P.octant = paths[p][0];
    P.level = (int)paths[p].size() - 1;
    path_verts(paths[p], P.v);
  }
  const int a = m.a;
  m.w.assign((size_t)m.P * a, 0.0);
  m.M.assign((size_t)m.P * a * a, 0.0);
  m.A.assign((size_t)m.P * 3 * a * a, 0.0);
  m.Aw.assign((size_t)m.P * 3 * a, 0.0);
  std::vector<double> nodes, wts;
  double psi[3];
  for (int p = 0; p < m.P; ++p) {
    patch_quadrature(m.patch[p], quadrature_order(m.patch[p].level, 4), nodes, wts);
    for (size_t k = 0; k < wts.size(); ++k) {
      const double* om = &nodes[3 * k];
      basis_values(m, p, om, psi);
      for (int i = 0; i < a; ++i) {
        m.w[p * a + i] += wts[k] * psi[i];
        for (int xi = 0; xi < 3; ++xi) m.Aw[(p * 3 + xi) * a + i] += wts[k] * om[xi] * psi[i];
        for (int j = 0; j < a; ++j) {
          double pp = wts[k] * psi[i] * psi[j];
          m.M[(p * a + i) * a + j] += pp;
          for (int xi = 0; xi < 3; ++xi) m.A[((p * 3 + xi) * a + i) * a + j] += pp * om[xi];
        }
      }
    }
  }
  return m;
}

namespace {
// Coefficients of the normalised associated Legendre recurrence, which depend
// on (n, m) only: the sectoral step sqrt((2m+1)/(2m)), the first off-sectoral
// factor sqrt(2m+3), and the three-term factors aa(n, m), bb(n, m) for
// n >= m + 2 (index m (N+1) + n).  Tabulated once per order instead of at
// every quadrature node; the values are the same expressions.
struct LegendreCoef {
  int N = 0;
  std::vector<double> step, first, aa, bb;
};

LegendreCoef legendre_coef(int N) {
  LegendreCoef c;
  c.N = N;
  c.step.assign(N + 1, 0.0);
  c.first.assign(N + 1, 0.0);
  c.aa.assign((size_t)(N + 1) * (N + 1), 0.0);
  c.bb.assign((size_t)(N + 1) * (N + 1), 0.0);
  for (int m = 0; m <= N; ++m) {
    if (m > 0) c.step[m] = std::sqrt((2.0 * m + 1.0) / (2.0 * m));
    c.first[m] = std::sqrt(2.0 * m + 3.0);
    for (int n = m + 2; n <= N; ++n) {
      c.aa[(size_t)m * (N + 1) + n] =
          std::sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
      c.bb[(size_t)m * (N + 1) + n] =
          std::sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
    }
  }
  return c;
}

void real_harmonics(const LegendreCoef& c, const double om[3], double* out) {
  // polar axis e_x: t = om_x, azimuthal plane (om_y, om_z)
  const int N = c.N;
  const double t = om[0];
  const double u = om[1], v = om[2];
  double cm = 1.0 / std::sqrt(4.0 * M_PI);  // Q_m^m (normalised, divided by sin^m)
  double re = 1.0, im = 0.0;                // (u + i v)^m
  for (int m = 0; m <= N; ++m) {
    if (m > 0) {
      cm *= c.step[m];
      double r2 = re * u - im * v;
      double i2 = re * v + im * u;
      re = r2;
      im = i2;
    }
    const double* aa = &c.aa[(size_t)m * (N + 1)];
    const double* bb = &c.bb[(size_t)m * (N + 1)];
    double qnm2 = 0.0, qnm1 = cm;
    for (int n = m; n <= N; ++n) {
      double q;
      if (n == m) {
        q = cm;
      } else if (n == m + 1) {
        q = c.first[m] * t * cm;
      } else {
        q = aa[n] * (t * qnm1 - bb[n] * qnm2);
      }
      if (n > m) {
        qnm2 = qnm1;
        qnm1 = q;
      }
      const int base = n * n + n;
      if (m == 0) {
        out[base] = q;
      } else {
        out[base + m] = M_SQRT2 * q * re;
        out[base - m] = M_SQRT2 * q * im;
      }
    }
  }
}
}  // namespace

void real_harmonics(int N, const double om[3], double* out) {
  real_harmonics(legendre_coef(N), om, out);
}

std::vector<double> x_table(const AngMesh& m, int N) {
  const int nm = (N + 1) * (N + 1);
  const int a = m.a;
  std::vector<double> X((size_t)m.P * a * nm, 0.0);
  const LegendreCoef c = legendre_coef(N);
  // Patches are independent: spread them over the host's cores.  Inside a
  // patch the harmonics are generated azimuthal order by azimuthal order for
  // all quadrature nodes at once (each node keeps its running sectoral value
  // and (u + i v)^m), so the entries of X that one order touches stay in the
  // first-level cache while the nodes stream past; every entry still sums its
  // node terms w_k Psi_i Y_j in node order, as the node-by-node loop did.
  std::atomic<int> next{0};
  auto work = [&] {
    std::vector<double> nodes, wts, T, U, V, CM, RE, IM, WP;
    double psi[3];
    for (int p; (p = next.fetch_add(1)) < m.P;) {
      patch_quadrature(m.patch[p], quadrature_order(m.patch[p].level, N), nodes, wts);
      const size_t K = wts.size();
      T.resize(K), U.resize(K), V.resize(K), CM.assign(K, 1.0 / std::sqrt(4.0 * M_PI));
      RE.assign(K, 1.0), IM.assign(K, 0.0), WP.resize(K * a);
      for (size_t k = 0; k < K; ++k) {
        const double* om = &nodes[3 * k];
        // polar axis e_x: t = om_x, azimuthal plane (om_y, om_z)
        T[k] = om[0], U[k] = om[1], V[k] = om[2];
        basis_values(m, p, om, psi);
        for (int i = 0; i < a; ++i) WP[k * a + i] = wts[k] * psi[i];
      }
      double* Xp = &X[(size_t)p * a * nm];
      for (int mo = 0; mo <= N; ++mo) {
        const double* aa = &c.aa[(size_t)mo * (N + 1)];
        const double* bb = &c.bb[(size_t)mo * (N + 1)];
        for (size_t k = 0; k < K; ++k) {
          if (mo > 0) {
            CM[k] *= c.step[mo];
            const double r2 = RE[k] * U[k] - IM[k] * V[k];
            const double i2 = RE[k] * V[k] + IM[k] * U[k];
            RE[k] = r2;
            IM[k] = i2;
          }
          const double t = T[k], cm = CM[k], re = RE[k], im = IM[k];
          const double* wp = &WP[k * a];
          double qnm2 = 0.0, qnm1 = cm;
          for (int n = mo; n <= N; ++n) {
            double q;
            if (n == mo) {
              q = cm;
            } else if (n == mo + 1) {
              q = c.first[mo] * t * cm;
            } else {
              q = aa[n] * (t * qnm1 - bb[n] * qnm2);
            }
            if (n > mo) {
              qnm2 = qnm1;
              qnm1 = q;
            }
            const int base = n * n + n;
            if (mo == 0) {
              for (int i = 0; i < a; ++i) Xp[(size_t)i * nm + base] += wp[i] * q;
            } else {
              const double yr = M_SQRT2 * q * re;
              const double yi = M_SQRT2 * q * im;
              for (int i = 0; i < a; ++i) {
                Xp[(size_t)i * nm + base + mo] += wp[i] * yr;
                Xp[(size_t)i * nm + base - mo] += wp[i] * yi;
              }
            }
          }
        }
      }
    }
  };
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 1;
  if (nt > 64) nt = 64;
  if ((int)nt > m.P) nt = (unsigned)m.P;
  if (nt <= 1) {
    work();
    return X;
  }
  std::vector<std::thread> ts;
  for (unsigned t = 0; t < nt; ++t) ts.emplace_back(work);
  for (auto& t : ts) t.join();
  return X;
}

double beam_weights(const AngMesh& m, const double om[3], double fac, double* out) {
  const int a = m.a;
  double total = 0.0;
  for (int q = 0; q < m.P; ++q) {
    const auto& V = m.patch[q].v;
    // om = sum_i lam_i V_i (Cramer's rule)
    auto det = [](const double* c0, const double* c1, const double* c2) {
      return c0[0] * (c1[1] * c2[2] - c1[2] * c2[1]) - c1[0] * (c0[1] * c2[2] - c0[2] * c2[1]) +
             c2[0] * (c0[1] * c1[2] - c0[2] * c1[1]);
    };
    const double D = det(V[0], V[1], V[2]);
    const double lam[3] = {det(om, V[1], V[2]) / D, det(V[0], om, V[2]) / D,
                           det(V[0], V[1], om) / D};
    const double lmax = std::max({std::fabs(lam[0]), std::fabs(lam[1]), std::fabs(lam[2])});
    if (std::min({lam[0], lam[1], lam[2]}) < -1e-12 * lmax) continue;
    int nz = 0, vi = -1;
    for (int i = 0; i < 3; ++i) {
      if (std::fabs(lam[i]) <= 1e-12 * lmax) ++nz;
      else vi = i;
    }
    double share = 1.0;
    if (nz == 1) {
      share = 0.5;
    } else if (nz == 2) {
      // interior angle at vertex vi between the great circles to the others
      const double* A = V[vi];
      const double* B = V[(vi + 1) % 3];
      const double* C = V[(vi + 2) % 3];
      double tb[3], tc[3];
      const double ab = A[0] * B[0] + A[1] * B[1] + A[2] * B[2];
      const double ac = A[0] * C[0] + A[1] * C[1] + A[2] * C[2];
      for (int e = 0; e < 3; ++e) {
        tb[e] = B[e] - ab * A[e];
        tc[e] = C[e] - ac * A[e];
      }
      const double cr[3] = {tb[1] * tc[2] - tb[2] * tc[1], tb[2] * tc[0] - tb[0] * tc[2],
                            tb[0] * tc[1] - tb[1] * tc[0]};
      const double dt = tb[0] * tc[0] + tb[1] * tc[1] + tb[2] * tc[2];
      share = std::atan2(std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]), dt) /
              (2.0 * M_PI);
    }
    double psi[3];
    basis_values(m, q, om, psi);
    for (int i = 0; i < a; ++i) out[q * a + i] = fac * share * psi[i];
    total += share;
  }
  return total;
}

Transfer build_transfer(const AngMesh& fine, const AngMesh& coarse) {
  Transfer t;
  const int a = fine.a;
  t.parent.assign(fine.P, -1);
  t.blk.assign((size_t)fine.P * a * a, 0.0);
  t.child_begin.assign(coarse.P, 0);
  t.child_end.assign(coarse.P, 0);
  int c = 0;
  for (int f = 0; f < fine.P; ++f) {
    const auto& fp = fine.patch[f].path;
    auto is_prefix = [&](int cc) {
      const auto& cp = coarse.patch[cc].path;
      return cp.size() <= fp.size() && std::equal(cp.begin(), cp.end(), fp.begin());
    };
    while (c < coarse.P && !is_prefix(c)) ++c;
    if (c >= coarse.P) throw std::runtime_error("angular meshes are not nested");
    if (t.child_end[c] == 0 && t.child_begin[c] == 0) t.child_begin[c] = f;
    t.parent[f] = c;
    t.child_end[c] = f + 1;
    if (a == 1) {
      t.blk[f] = 1.0;
    } else {
      for (int k = 0; k < 3; ++k) {
        double val[3];
        basis_values(coarse, c, fine.patch[f].v[k], val);
        for (int d = 0; d < 3; ++d) t.blk[(f * 3 + k) * 3 + d] = val[d];
      }
    }
  }
  return t;
}

Q1 build_q1(int dim, const double hin[3]) {
  Q1 q;
  q.dim = dim;
  q.s = 1 << dim;
  for (int e = 0; e < 3; ++e) q.h[e] = e < dim ? hin[e] : 1.0;
  const int s = q.s;
  auto m1 = [&](int e, int i, int j) { return q.h[e] / 6.0 * (i == j ? 2.0 : 1.0); };
  auto g1 = [](int i, int) { return i == 0 ? -0.5 : 0.5; };
  auto bit = [](int n, int e) { return (n >> e) & 1; };
  q.N.assign(s * s, 0.0);
  q.V.assign(dim * s * s, 0.0);
  q.Fown.assign(2 * dim * s * s, 0.0);
  q.Fnb.assign(2 * dim * s * s, 0.0);
  q.mu.assign(s, 0.0);
  q.mf.assign(2 * dim * s, 0.0);
  q.facemass.assign(dim * (s / 2) * (s / 2), 0.0);
  for (int l = 0; l < s; ++l) {
    double vol = 1.0;
    for (int e = 0; e < dim; ++e) vol *= q.h[e] / 2.0;
    q.mu[l] = vol;
    for (int i = 0; i < s; ++i) {
      double nn = 1.0;
      for (int e = 0; e < dim; ++e) nn *= m1(e, bit(l, e), bit(i, e));
      q.N[l * s + i] = nn;
      for (int xi = 0; xi < dim; ++xi) {
        double vv = g1(bit(l, xi), bit(i, xi));
        double ff = 1.0;
        for (int e = 0; e < dim; ++e)
          if (e != xi) ff *= m1(e, bit(l, e), bit(i, e));
        q.V[(xi * s + l) * s + i] = vv * ff;
        for (int side = 0; side < 2; ++side) {
          int f = 2 * xi + side;
          if (bit(l, xi) == side && bit(i, xi) == side) q.Fown[(f * s + l) * s + i] = ff;
          if (bit(l, xi) == side && bit(i, xi) == 1 - side) q.Fnb[(f * s + l) * s + i] = ff;
        }
      }
    }
    for (int xi = 0; xi < dim; ++xi)
      for (int side = 0; side < 2; ++side) {
        double a = 1.0;
        for (int e = 0; e < dim; ++e)
          if (e != xi) a *= q.h[e] / 2.0;
        q.mf[(2 * xi + side) * s + l] = bit(l, xi) == side ? a : 0.0;
      }
  }
  const int hs = s / 2;
  for (int xi = 0; xi < dim; ++xi)
    for (int jp = 0; jp < hs; ++jp)
      for (int j = 0; j < hs; ++j) {
        int l = face_node(jp, xi, 0), i = face_node(j, xi, 0);
        double ff = 1.0;
        for (int e = 0; e < dim; ++e)
          if (e != xi) ff *= m1(e, bit(l, e), bit(i, e));
        q.facemass[(xi * hs + jp) * hs + j] = ff;
      }
  return q;
}

bool invert(int n, const double* A, double* Ainv) {
  std::vector<double> M(A, A + (size_t)n * n);
  std::vector<double> I((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(M[r * n + col]) > std::fabs(M[piv * n + col])) piv = r;
    if (M[piv * n + col] == 0.0) return false;
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(M[col * n + k], M[piv * n + k]);
        std::swap(I[col * n + k], I[piv * n + k]);
      }
    double d = 1.0 / M[col * n + col];
    for (int k = 0; k < n; ++k) {
      M[col * n + k] *= d;
      I[col * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = M[r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        M[r * n + k] -= f * M[col * n + k];
        I[r * n + k] -= f * I[col * n + k];
      }
    }
  }
  std::memcpy(Ainv, I.data(), sizeof(double) * n * n);
  return true;
}

}  // namespace amgt
