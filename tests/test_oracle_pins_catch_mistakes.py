"""Planted mistakes: each case plants one plausible mistake into the oracle (on
the CPU, for the duration of that case only, through monkeypatch) and checks
that the pin named beside it then fails.  A pin that still passed with the
mistake planted would not pin the function; these cases show that a dropped
term, a wrong sign, index, operand or order in each oracle function is caught
by a pin fixed by the paper or the mathematics (dense LU, closed forms,
LAPACK, scipy, the paper's printed mesh sizes, finite differences).

The Krylov oracles (GMRES, BiCGStab) are pinned on their returned solution
against LAPACK; the cases below show that an update along the wrong
directions or a dropped stabilisation step fails those pins.  (A mistake that
only slows the iteration -- a Givens rotation of the wrong sign, say, which
each restart's true residual corrects -- leaves the answer, and the pins,
unchanged.)
"""
import numpy as np
import pytest

import test_oracle_adjoint as PA
import test_oracle_angular as PG
import test_oracle_beam as PB
import test_oracle_harmonics_spatial as PH
import test_oracle_materials as PM
import test_oracle_transport as PT
import test_oracle_vcycle as PV
import test_oracle_bicgstab as PK
from oracle import adjoint, angular, bicgstab, gmres, harmonics, multigrid, spatial, transport


# --------------------------------------------------------------- V-cycle
def _cycle(drop_pre=False, drop_post=False, restrict_f=False, subtract=False,
           residual_L=False, restrict_l2=False):
    """The cycle of Fig. lmg with one step changed."""
    def vcycle(self, f, k=0, phi=None):
        T = self.levels[k]
        if phi is None:
            phi = np.zeros_like(f)
        if k == len(self.levels) - 1:
            return multigrid.coarse_gs(T, f, phi, self.coarse_sweeps)
        phi = self.smooth(phi, f, k, 0 if drop_pre else self.nu_pre)
        r = f - (T.apply_L(phi) if residual_L else T.apply_A(phi))
        src = f if restrict_f else r
        if restrict_l2:                        # L2 projection instead of P^T
            Pk = self.P[k]
            fc = np.linalg.solve(Pk.T @ Pk, (src @ Pk).T).T
        else:
            fc = self.restrict(src, k)
        phic = self.vcycle(fc, k + 1, None)
        phi = phi - self.prolong(phic, k) if subtract else phi + self.prolong(phic, k)
        return self.smooth(phi, f, k, 0 if drop_post else self.nu_post)
    return vcycle


def _smooth_without_scatter(self, phi, f, k, nu):
    T = self.levels[k]
    for _ in range(nu):
        phi = T.sweep(f)
    return phi


def _two_grid():
    PV.test_two_grid_error_propagator(1, 1, (6, 3))


VCYCLE = {
    "post-smoothing dropped": (lambda mp: mp.setattr(multigrid.Hierarchy, "vcycle", _cycle(drop_post=True)), _two_grid),
    "pre-smoothing dropped": (lambda mp: mp.setattr(multigrid.Hierarchy, "vcycle", _cycle(drop_pre=True)), _two_grid),
    "f restricted instead of the residual": (lambda mp: mp.setattr(multigrid.Hierarchy, "vcycle", _cycle(restrict_f=True)), _two_grid),
    "coarse correction subtracted": (lambda mp: mp.setattr(multigrid.Hierarchy, "vcycle", _cycle(subtract=True)), _two_grid),
    "residual with L instead of A": (lambda mp: mp.setattr(multigrid.Hierarchy, "vcycle", _cycle(residual_L=True)), _two_grid),
    "restriction by L2 projection instead of P^T": (lambda mp: mp.setattr(multigrid.Hierarchy, "vcycle", _cycle(restrict_l2=True)),
                                                    PV.test_cycle_without_smoothing_is_coarse_correction),
    "smoother without the scatter source": (lambda mp: mp.setattr(multigrid.Hierarchy, "smooth", _smooth_without_scatter), _two_grid),
    "coarse level at the fine scatter order": (
        lambda mp: mp.setattr(multigrid, "Transport",
                              lambda prob, am, N=None: transport.Transport(prob, am, prob["mg"]["Nr"][0])),
        _two_grid),
}


# --------------------------------------------------------- coarse Gauss-Seidel
def _coarse_gs(jacobi=False, no_self=False, reverse=False, one_shape=False, nb_sign=1.0):
    """Block Gauss-Seidel of Sec. 4.2 with one step changed."""
    def coarse_gs(T, f, phi, nsweeps):
        s, a = T.s, T.a
        fb = T.to_blocks(f)
        xb = T.to_blocks(phi).copy()
        Sfs = [T.angular_scatter_matrix(m) for m in range(T.nshape)]
        N = T.cell.N
        for _ in range(nsweeps):
            start = xb.copy()
            for d in range(T.ndir):
                order = T.sweep_order(d)
                for c in (order[::-1] if reverse else order):
                    for q in T.patches_of(d):
                        rhs = fb[c, q].copy()
                        for fc in range(2 * T.dim):
                            nb = T.neighbour(c, fc)
                            if nb >= 0 and not T.outflow[fc, q]:
                                rhs -= nb_sign * (T.U[fc, q] @ xb[nb, q])
                        xc = (start if jacobi else xb)[c].reshape(T.P, s, a)
                        Sf = Sfs[0 if one_shape else T.fid[c]]
                        src = np.zeros((s, a))
                        for p in range(T.P):
                            if p != q:
                                src += N @ xc[p] @ Sf[q * a:(q + 1) * a, p * a:(p + 1) * a].T
                        rhs += T.sigma_s[c] * src.reshape(-1)
                        Sqq = Sf[q * a:(q + 1) * a, q * a:(q + 1) * a]
                        Amat = T.block(c, q) - (0.0 if no_self else T.sigma_s[c]) * np.kron(N, Sqq)
                        xb[c, q] = np.linalg.solve(Amat, rhs)
        return T.from_blocks(xb)
    return coarse_gs


GS = {
    "other patches of the cell from the sweep's start (Jacobi)": (
        lambda mp: mp.setattr(multigrid, "coarse_gs", _coarse_gs(jacobi=True)),
        PT.test_coarse_gs_block_equation_holds),
    "self-scatter left out of the block solve": (
        lambda mp: mp.setattr(multigrid, "coarse_gs", _coarse_gs(no_self=True)),
        PT.test_coarse_gs_fixed_point_and_convergence),
    "cells visited downwind first": (
        lambda mp: mp.setattr(multigrid, "coarse_gs", _coarse_gs(reverse=True)),
        PT.test_coarse_gs_block_equation_holds),
    "one moment shape for every material": (
        lambda mp: mp.setattr(multigrid, "coarse_gs", _coarse_gs(one_shape=True)),
        PM.test_coarse_gs_fixed_point_with_two_shapes),
    "upwind coupling with the wrong sign": (
        lambda mp: mp.setattr(multigrid, "coarse_gs", _coarse_gs(nb_sign=-1.0)),
        PT.test_coarse_gs_fixed_point_and_convergence),
}


# ------------------------------------------------------------- transport
def _sweep_without_y_faces(self, b, patches=None):
    bb = self.to_blocks(b)
    psi = np.zeros_like(bb)
    for d in range(self.ndir):
        qs = self.patches_of(d)
        for c in self.sweep_order(d):
            rhs = bb[c, qs].copy()
            for f in range(2 * self.dim):
                nb = self.neighbour(c, f)
                if nb < 0 or f in (2, 3):
                    continue
                rhs -= np.einsum("qij,qj->qi", self.U[f, qs], psi[nb, qs])
            psi[c, qs] = np.linalg.solve(self.block(c, qs), rhs[..., None])[..., 0]
    return self.from_blocks(psi)


def _apply_L_neighbour_sign(self, x, cells=None):
    xb = self.to_blocks(x)
    yb = np.zeros_like(xb)
    for c in range(self.C):
        yb[c] = np.einsum("qij,qj->qi", self.block(c, slice(None)), xb[c])
        for f in range(2 * self.dim):
            nb = self.neighbour(c, f)
            if nb >= 0:
                yb[c] -= np.einsum("qij,qj->qi", self.U[f], xb[nb])
    return self.from_blocks(yb)


def _scatter_without_mass(self, x, cells=None):
    Phi = x @ self.X
    Frow = np.repeat(self.Ftab[self.fid], self.s, axis=0)
    Yang = (Phi * Frow) @ self.X.T
    return np.repeat(self.sigma_s, self.s)[:, None] * Yang


def _wrap_init(cls, after):
    orig = cls.__init__

    def init(self, *a, **k):
        orig(self, *a, **k)
        after(self)
    return init


def _downwind(mp):
    mp.setattr(angular.AngularMesh, "__init__",
               _wrap_init(angular.AngularMesh, lambda am: setattr(am, "signs", -am.signs)))


def _2d_directions_from_y_and_z(mp):
    def after(T):
        if T.dim == 2:
            T.pdir = np.array([2 * ((o >> 1) & 1) + (o & 1) for o in T.am.octant])
    mp.setattr(transport.Transport, "__init__", _wrap_init(transport.Transport, after))


def _with_prob(method, change):
    """The method run on the problem with one entry changed."""
    def run(self, *a, **k):
        saved = self.prob
        self.prob = change(dict(saved))
        try:
            return method(self, *a, **k)
        finally:
            self.prob = saved
    return run


def _source_without_4pi(mp):
    def change(p):
        p["q"] = 4.0 * np.pi * np.asarray(p["q"], dtype=np.float64)
        return p
    mp.setattr(transport.Transport, "source", _with_prob(transport.Transport.source, change))


def _inflow_sign(mp):
    def change(p):
        p["boundary"] = [(k, -v if k == 1 else v) for k, v in p["boundary"]]
        return p
    mp.setattr(transport.Transport, "source", _with_prob(transport.Transport.source, change))


def _degree_shift(mp):
    orig = harmonics.degree_of_index
    mp.setattr(harmonics, "degree_of_index",
               lambda N: np.minimum(orig(N) + 1, N))


def _with_fid0(method):
    def run(self, *a, **k):
        saved = self.fid
        self.fid = np.zeros_like(saved)
        try:
            return method(self, *a, **k)
        finally:
            self.fid = saved
    return run


def _infinite_medium():
    PT.test_infinite_medium_closed_form(2, (3, 2), "lin")


def _sweep_pin():
    PT.test_sweep_is_exact_inverse_of_L(*PT.CASES[0])


TRANSPORT = {
    "sweep without the y-face inflow": (lambda mp: mp.setattr(transport.Transport, "sweep", _sweep_without_y_faces), _sweep_pin),
    "L's upwind coupling with the wrong sign": (lambda mp: mp.setattr(transport.Transport, "apply_L", _apply_L_neighbour_sign), _sweep_pin),
    "downwind instead of upwind face fluxes": (_downwind, _sweep_pin),
    "2D sweep directions from the y and z signs": (_2d_directions_from_y_and_z, _sweep_pin),
    "collision with sigma_s instead of sigma_t": (
        lambda mp: mp.setattr(transport.Transport, "block",
                              lambda self, c, q: self.K0[q] + self.sigma_s[c] * self.B[q]),
        _infinite_medium),
    "scatter without the spatial mass matrix": (
        lambda mp: mp.setattr(transport.Transport, "scatter", _scatter_without_mass),
        lambda: PT.test_gmres_matches_dense_lu(*PT.CASES[0])),
    "Legendre moment f_n applied at degree n + 1": (_degree_shift, PT.test_scatter_matrix_equals_legendre_double_integral),
    "isotropic source without 1/(4 pi)": (_source_without_4pi, _infinite_medium),
    "isotropic inflow with the wrong sign": (_inflow_sign, _infinite_medium),
    "scalar flux without the angular weights": (
        lambda mp: mp.setattr(transport.Transport, "scalar_flux", lambda self, psi: psi.sum(axis=1)),
        _infinite_medium),
    "scatter of every cell with material 0's shape": (
        lambda mp: mp.setattr(transport.Transport, "scatter",
                              _with_fid0(transport.Transport.scatter)),
        lambda: PM.test_two_shape_solution_matches_dense_lu(2, (3, 3), 1)),
}


# ---------------------------------------------------------------- angular
def _child_vertices_wrong_pair(verts, c):
    a, b, cc = verts
    ab = angular._unit(a + b)
    bc = angular._unit(b + cc)
    ca = angular._unit(cc + a)
    return np.array([(a, ab, ca), (ab, b, ca), (ca, bc, cc), (ab, bc, ca)][c])


def _basis_without_projection(verts, octant, basis, omega):
    omega = np.asarray(omega, dtype=np.float64)
    if basis == "const":
        return np.ones(omega.shape[:-1] + (1,))
    U = angular.flat_vertices(verts).T
    lam = np.linalg.solve(U, omega.reshape(-1, 3).T).T
    return lam.reshape(omega.shape[:-1] + (3,))


def _prolongation_transposed_block(fine, coarse):
    P = np.zeros((fine.nadof, coarse.nadof))
    index = {p: i for i, p in enumerate(coarse.paths)}
    for f, path in enumerate(fine.paths):
        c = next(index[path[:k]] for k in range(len(path), 0, -1) if path[:k] in index)
        if fine.basis == "const":
            P[f, c] = 1.0
        else:
            vals = angular.basis_eval(coarse.verts[c], coarse.octant[c], "lin", fine.verts[f])
            P[f * 3:(f + 1) * 3, c * 3:(c + 1) * 3] = vals.T
    return P


def _aniso_target_095(verts, axis, lmax):
    m = max(float(np.dot(v, axis)) for v in verts)
    for t, lim in enumerate((0.95, 0.9, 0.8, 0.6)):
        if m > lim:
            return max(lmax - t, 0)
    return max(lmax - 4, 0)


ANGULAR = {
    "gnomonic Jacobian without the plane distance": (
        lambda mp: mp.setattr(angular, "H_PLANE", 1.0), lambda: PG.test_uniform_counts_and_areas(1)),
    "daughter 1 built on the wrong edge midpoint": (
        lambda mp: mp.setattr(angular, "child_vertices", _child_vertices_wrong_pair),
        lambda: PG.test_uniform_counts_and_areas(1)),
    "Lin basis without the central projection": (
        lambda mp: mp.setattr(angular, "basis_eval", _basis_without_projection),
        PG.test_lin_nodal_and_partition_of_unity),
    "prolongation block transposed": (
        lambda mp: mp.setattr(angular, "prolongation", _prolongation_transposed_block),
        lambda: PG.test_prolongation_exact_and_galerkin("lin")),
    "first refinement band at 0.95 instead of 0.97": (
        lambda mp: mp.setattr(angular, "aniso_target", _aniso_target_095),
        PG.test_aniso_counts_match_paper),
}


# ------------------------------------------------- harmonics and Q1 cell
def _harmonics_without_sqrt2(mp):
    orig = harmonics.real_sph_harm

    def Y(N, om):
        out = orig(N, om)
        o = np.arange(harmonics.nmoments(N)) - harmonics.degree_of_index(N) * (harmonics.degree_of_index(N) + 1)
        out[..., o != 0] /= np.sqrt(2.0)
        return out
    mp.setattr(harmonics, "real_sph_harm", Y)


def _gauss_degree1(n):
    return np.array([1.0, 3.0, 5.0]) / 6.0, np.full(3, 1.0 / 3.0)


def _nb_trace_is_own(mp):
    mp.setattr(spatial.Q1Cell, "__init__",
               _wrap_init(spatial.Q1Cell, lambda c: setattr(c, "Fnb", c.Fown.copy())))


LOCAL = {
    "real harmonics without sqrt(2) for o != 0": (_harmonics_without_sqrt2, PH.test_real_harmonics_match_scipy),
    "Q1 matrices from a rule exact only for degree 1": (
        lambda mp: mp.setattr(spatial, "_gauss01", _gauss_degree1), PH.test_q1_2d_closed_forms),
    "neighbour's trace replaced by the own trace": (_nb_trace_is_own, PH.test_q1_2d_closed_forms),
    "Q1 derivative with the wrong sign": (
        lambda mp: mp.setattr(spatial.Q1Cell, "_dl", lambda self, a, h: (1.0 / h) if a == 0 else (-1.0 / h)),
        PH.test_q1_2d_closed_forms),
}


# -------------------------------------------------------- beams and adjoint
def _edge_share_one(mp):
    orig = transport.beam_weights

    def wb(am, om):
        out = orig(am, om)
        if np.count_nonzero(out.any(axis=1)) == 2:      # the direction lies on an edge
            out = 2.0 * out
        return out
    mp.setattr(transport, "beam_weights", wb)


def _beam_cosine_dropped(mp):
    orig = transport.Transport._general_beam

    def gb(self, fb, f, val):
        om = np.asarray(val[1:4], dtype=np.float64)
        om = om / np.linalg.norm(om)
        n = np.zeros(3)
        n[f // 2] = 2.0 * (f % 2) - 1.0
        v = list(val)
        v[0] = float(val[0]) / abs(om @ n)
        return orig(self, fb, f, v)
    mp.setattr(transport.Transport, "_general_beam", gb)


def _general_cap(name):
    e = dict(PB._general_directions())[name]
    return lambda: PB.test_general_beam_weights_are_the_limit_of_a_shrinking_cap(
        "lin", angular.uniform_paths(2), name, e)


def _reversed_keeps(attr):
    def plant(mp):
        mp.setattr(adjoint.ReversedMesh, "__init__",
                   _wrap_init(adjoint.ReversedMesh, lambda m: setattr(m, attr, getattr(m._am, attr))))
    return plant


def _dsigt_sign(mp):
    orig = adjoint.gradients
    mp.setattr(adjoint, "gradients", lambda T, psi, lam: (lambda g: (-g[0], g[1], g[2]))(orig(T, psi, lam)))


BEAM_ADJOINT = {
    "beam share at a vertex from twice its angle": (
        lambda mp: mp.setattr(transport, "_vertex_angle",
                              (lambda f: lambda A, B, C: 2.0 * f(A, B, C))(transport._vertex_angle)),
        _general_cap("vertex1")),
    "beam share 1 on an edge": (_edge_share_one, _general_cap("edge")),
    "oblique beam without its cosine": (
        _beam_cosine_dropped,
        lambda: PB.test_general_beam_source_total_is_its_incident_current(2, (5, 7), 0, (0.23, 0.61, 0.0, 0.0))),
    "reversed mesh keeps A^xi": (_reversed_keeps("A"),
                                 lambda: PA.test_reversed_direction_operator_is_the_transpose(*PA.CASES[0])),
    "reversed mesh keeps the octant bits": (_reversed_keeps("octant"),
                                            lambda: PA.test_reversed_direction_sweep_inverts_the_transpose(*PA.CASES[0])),
    "sigma_t gradient with the wrong sign": (_dsigt_sign,
                                            lambda: PA.test_gradients_match_central_differences(*PA.CASES[2])),
}


# ------------------------------------------------------------------ Krylov
def _gmres(update_with_V=False):
    """Right-preconditioned restarted GMRES(m) with CGS2 and Givens rotations
    (the oracle's method) with one step changed."""
    def run(apply_A, b, apply_M, tol, restart=20, maxit=1000, x0=None):
        x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
        bnorm = np.linalg.norm(b)
        its = 0
        m = restart
        while True:
            r = b - apply_A(x)
            beta = np.linalg.norm(r)
            rel = beta / bnorm
            if rel < tol or its >= maxit:
                return x, its, [], rel
            V, Z = [r / beta], []
            H = np.zeros((m + 1, m))
            cs, sn, g = np.zeros(m), np.zeros(m), np.zeros(m + 1)
            g[0] = beta
            k = 0
            for j in range(m):
                z = apply_M(V[j])
                w = apply_A(z).reshape(-1)
                Vm = np.stack([v.reshape(-1) for v in V])
                h = Vm @ w
                w = w - Vm.T @ h
                h2 = Vm @ w
                w = w - Vm.T @ h2
                hn = np.linalg.norm(w)
                H[:j + 1, j] = h + h2
                H[j + 1, j] = hn
                Z.append(z)
                for i in range(j):
                    t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                    H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                    H[i, j] = t
                den = np.hypot(H[j, j], H[j + 1, j])
                cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
                H[j, j], H[j + 1, j] = den, 0.0
                g[j + 1] = -sn[j] * g[j]
                g[j] = cs[j] * g[j]
                its += 1
                k = j + 1
                if abs(g[j + 1]) / bnorm < tol or its >= maxit or hn == 0.0:
                    break
                V.append((w / hn).reshape(b.shape))
            y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
            for i in range(k):
                x = x + y[i] * (V[i] if update_with_V else Z[i])
    return run


def _bicgstab_without_stabilisation_update(apply_A, b, apply_M, tol, maxit=1000, x0=None):
    """BiCGStab whose iterate misses the minimal-residual step omega M^-1 s
    (the residual recursion keeps it)."""
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    r = b - apply_A(x)
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    its = 0
    while its < maxit and np.linalg.norm(r) / bnorm >= tol:
        its += 1
        rho = np.vdot(rhat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = apply_M(p)
        v = apply_A(ph)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        sh = apply_M(s)
        t = apply_A(sh)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * ph
        r = s - omega * t
        rho_old = rho
    return x, its, [], np.linalg.norm(b - apply_A(x)) / bnorm


def _gmres_pin():
    PT.test_gmres_matches_dense_lu(*PT.CASES[0])


def _bicgstab_pin():
    PK.test_sweep_preconditioned_matches_dense_lu(2, (3, 2), 1, "lin")


KRYLOV = {
    "GMRES update along the unpreconditioned directions": (
        lambda mp: mp.setattr(gmres, "gmres", _gmres(update_with_V=True)), _gmres_pin),
    "BiCGStab iterate without the stabilisation step": (
        lambda mp: mp.setattr(bicgstab, "bicgstab", _bicgstab_without_stabilisation_update),
        _bicgstab_pin),
}


def test_the_krylov_mutant_without_a_mistake_passes_the_pins(monkeypatch):
    """The GMRES copy above, with no step changed, passes the pin: the
    failures above come from the planted mistakes alone."""
    monkeypatch.setattr(gmres, "gmres", _gmres())
    _gmres_pin()


ALL = {**VCYCLE, **GS, **TRANSPORT, **ANGULAR, **LOCAL, **BEAM_ADJOINT, **KRYLOV}


@pytest.mark.parametrize("name", list(ALL))
def test_pin_fails_with_the_mistake_planted(name, monkeypatch):
    plant, pin = ALL[name]
    with monkeypatch.context() as mp:
        plant(mp)
        with pytest.raises(AssertionError):
            pin()
