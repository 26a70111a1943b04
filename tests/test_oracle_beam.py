"""Pins of the oracle's pencil-beam boundary source (Sec. 5.4, Dirac boundary
data in the DG weak form): the beam term is the limit of a uniform inflow over
a shrinking cap around the beam direction (integrated here by polar quadrature
on the sphere, patch by patch), its total is the incident current S * |face|,
and the solved flux obeys global particle balance, the mirror symmetry of the
set-up and, without scatter, stays on the patches holding the beam direction."""
import numpy as np
import pytest

import workloads as W
from oracle import angular, gmres, transport


def _owner(am, omega):
    for q in range(am.P):
        if np.linalg.solve(am.verts[q].T, omega).min() > -1e-13:
            return q
    raise AssertionError("direction in no patch")


def _cap_term(am, e, eps, S=1.0, nth=6, nph=8):
    """-int_{D_q} (Omega.n) Psi_m psi_b for the uniform inflow psi_b = c on
    the cap angle(Omega, e) < eps, c fixed by int_cap (Omega.e) psi_b = S,
    n = -e.  Polar Gauss quadrature about e, each of the four quarters split
    by the coordinate planes through e integrated on its own."""
    t1 = np.roll(e, 1)
    t2 = np.cross(e, t1)
    c = S / (np.pi * np.sin(eps) ** 2)
    g, wg = np.polynomial.legendre.leggauss(nth)
    gp, wgp = np.polynomial.legendre.leggauss(nph)
    out = np.zeros((am.P, am.a))
    for k in range(4):
        for th, wth in zip(0.5 * eps * (g + 1), 0.5 * eps * wg):
            for ph, wph in zip(0.25 * np.pi * (gp + 1 + 2 * k), 0.25 * np.pi * wgp):
                om = np.cos(th) * e + np.sin(th) * (np.cos(ph) * t1 + np.sin(ph) * t2)
                q = _owner(am, om)
                psi = angular.basis_eval(am.verts[q], am.octant[q], am.basis, om)
                out[q] += c * wth * wph * np.sin(th) * np.cos(th) * psi
    return out


MESHES = [("lin", angular.uniform_paths(0)), ("lin", angular.uniform_paths(2)),
          ("const", angular.uniform_paths(1)),
          ("lin", angular.aniso_paths(3, (1.0, 0.0, 0.0)))]


@pytest.mark.parametrize("basis,paths", MESHES, ids=["lin0", "lin2", "const1", "aniso3x"])
@pytest.mark.parametrize("e", [(1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (0.0, 0.0, 1.0)])
def test_beam_weights_are_the_limit_of_a_shrinking_cap(basis, paths, e):
    am = angular.AngularMesh(paths, basis)
    e = np.array(e)
    wb = transport.beam_weights(am, e)
    f1 = _cap_term(am, e, 8e-4)
    f2 = _cap_term(am, e, 4e-4)
    assert np.abs(f2 - wb).max() < 1e-2
    assert np.abs(f2 - wb).max() > 1e-6 or basis == "const"
    assert np.abs((2 * f2 - f1) - wb).max() < 1e-6
    assert abs(wb.sum() - 1.0) < 1e-14
    assert np.count_nonzero(wb.any(axis=1)) == 4


def _beam_problem(dim, nc, level, face, S, ss_frac, basis="lin", N=4, g=0.8):
    C = int(np.prod(nc))
    bnd = [(0, 0.0)] * (2 * dim)
    bnd[face] = (2, S)
    st = np.full(C, 2.0)
    return W.problem(dim, nc, st, ss_frac * st, N, W.hg_moments(g, N), np.zeros(C), level,
                     basis=basis, boundary=bnd)


def _T(prob):
    am = angular.AngularMesh(angular.uniform_paths(prob["level"]), prob["basis"])
    return transport.Transport(prob, am)


@pytest.mark.parametrize("dim,nc,level,face,basis", [
    (2, (3, 4), 1, 0, "lin"), (2, (4, 2), 0, 3, "const"), (3, (2, 2, 3), 0, 5, "lin")])
def test_beam_source_total_is_the_incident_current(dim, nc, level, face, basis):
    S = 1.7
    prob = _beam_problem(dim, nc, level, face, S, 0.5, basis)
    T = _T(prob)
    xi = face // 2
    area = np.prod([prob["hi"][e] - prob["lo"][e] for e in range(dim) if e != xi])
    f = T.source()
    assert abs(f.sum() - S * area) < 1e-13 * S * area
    assert (f >= -1e-15).all()


def _leak_and_absorption(T, psi):
    s, a = T.s, T.a
    leak = 0.0
    for c in range(T.C):
        blk = psi[c * s:(c + 1) * s].reshape(s, T.P, a)
        for f in range(2 * T.dim):
            if T.neighbour(c, f) >= 0:
                continue
            xi, side = divmod(f, 2)
            for q in range(T.P):
                if T.outflow[f, q]:
                    leak += T.cell.mf[f] @ blk[:, q, :] @ ((2.0 * side - 1.0) * T.am.Aw[q, xi])
    phis = T.scalar_flux(psi)
    absn = sum((T.sigma_t[c] - T.sigma_s[c]) * (T.cell.mu @ phis[c * s:(c + 1) * s])
               for c in range(T.C))
    return leak, absn


@pytest.mark.parametrize("dim,nc,level,face", [(2, (5, 4), 1, 0), (3, (2, 3, 2), 0, 4)])
def test_beam_solution_balances_the_incident_current(dim, nc, level, face):
    S = 1.0
    prob = _beam_problem(dim, nc, level, face, S, 0.8)
    T = _T(prob)
    x, _, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 400)
    assert rel < 1e-13
    leak, absn = _leak_and_absorption(T, x)
    area = np.prod([prob["hi"][e] - prob["lo"][e] for e in range(dim) if e != face // 2])
    assert abs(leak + absn - S * area) < 1e-11 * S * area
    assert leak > 0 and absn > 0


def test_beam_solution_is_mirror_symmetric_across_the_beam_axis():
    """Beam on the whole low-x edge of the unit square, vacuum elsewhere: the
    set-up is symmetric under y -> 1 - y, so are the cell averages of the
    scalar flux."""
    nx, ny = 4, 6
    prob = _beam_problem(2, (nx, ny), 1, 0, 1.0, 0.9, N=6, g=0.9)
    T = _T(prob)
    x, _, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 400)
    phis = T.scalar_flux(x).reshape(T.C, T.s) @ T.cell.mu
    avg = phis.reshape(ny, nx)
    assert np.abs(avg - avg[::-1]).max() < 1e-11 * np.abs(avg).max()


def test_unscattered_beam_stays_on_its_patches():
    prob = _beam_problem(2, (4, 3), 1, 0, 1.0, 0.0)
    T = _T(prob)
    x = T.sweep(T.source())
    hold = transport.beam_weights(T.am, np.array([1.0, 0.0, 0.0])).any(axis=1)
    blk = x.reshape(T.nsdof, T.P, T.a)
    assert np.abs(blk[:, ~hold]).max() == 0.0
    assert np.abs(blk[:, hold]).max() > 0.1


def test_beam_in_the_reversed_direction_mesh_is_the_same_physical_beam():
    """A mesh with every direction reversed holds -D_q in patch q; a beam on
    the low-x face still travels along +x, so the reversed problem's solution
    is the forward one with each patch relabelled to its antipode (octant
    bits flipped, same child path)."""
    from oracle import adjoint as oadj
    prob = _beam_problem(2, (4, 3), 1, 0, 1.0, 0.7)
    am = angular.AngularMesh(angular.uniform_paths(1), "lin")
    T = transport.Transport(prob, am)
    Tr = transport.Transport(prob, oadj.ReversedMesh(am))
    x, _, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 400)
    xr, _, _, relr = gmres.gmres(Tr.apply_A, Tr.source(), Tr.sweep, 1e-13, 20, 400)
    index = {p: i for i, p in enumerate(am.paths)}
    anti = [index[(p[0] ^ 7,) + tuple(p[1:])] for p in am.paths]
    perm = np.concatenate([np.arange(q * am.a, q * am.a + am.a) for q in anti])
    assert np.linalg.norm(xr[:, perm] - x) < 1e-11 * np.linalg.norm(x)


# ---------------------------------------------------------------- general beam
def _sector_edges(am, e, t1, t2):
    """Azimuths (about e, in the frame t1, t2) of the patch edges through e:
    the sector boundaries of a small cap around e."""
    phis = []
    for q in range(am.P):
        V = am.verts[q]
        lam = np.linalg.solve(V.T, e)
        if lam.min() < -1e-12:
            continue
        zero = np.abs(lam) <= 1e-12 * np.abs(lam).max()
        others = [V[i] for i in range(3) if zero[i]]  # e lies on edges to these... 
        if zero.sum() == 1:                            # on the edge opposite the zero
            i = int(np.argmax(zero))
            ends = [V[(i + 1) % 3], V[(i + 2) % 3]]
        elif zero.sum() == 2:                          # at the vertex with lam != 0
            i = int(np.argmax(~zero))
            ends = [V[(i + 1) % 3], V[(i + 2) % 3]]
        else:
            continue
        for B in ends:
            t = B - (B @ e) * e
            if np.linalg.norm(t) < 1e-9:
                continue
            phis.append(np.arctan2(t @ t2, t @ t1) % (2 * np.pi))
            if zero.sum() == 1:
                phis.append((phis[-1] + np.pi) % (2 * np.pi))
    return sorted(set(np.round(phis, 12)))


def _cap_term_general(am, e, eps, S=1.0, nth=6, nph=8):
    """As _cap_term, for any direction e: the cap is cut into the sectors
    between the patch edges through e, each integrated on its own."""
    t1 = np.cross(e, [0.3, 0.5, 0.7])
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(e, t1)
    cuts = _sector_edges(am, e, t1, t2)
    if not cuts:
        cuts = [0.0]
    bounds = cuts + [cuts[0] + 2 * np.pi]
    c = S / (np.pi * np.sin(eps) ** 2)
    g, wg = np.polynomial.legendre.leggauss(nth)
    gp, wgp = np.polynomial.legendre.leggauss(nph)
    out = np.zeros((am.P, am.a))
    for p0, p1 in zip(bounds[:-1], bounds[1:]):
        for th, wth in zip(0.5 * eps * (g + 1), 0.5 * eps * wg):
            for ph, wph in zip(p0 + 0.5 * (p1 - p0) * (gp + 1), 0.5 * (p1 - p0) * wgp):
                om = np.cos(th) * e + np.sin(th) * (np.cos(ph) * t1 + np.sin(ph) * t2)
                q = _owner(am, om)
                psi = angular.basis_eval(am.verts[q], am.octant[q], am.basis, om)
                out[q] += c * wth * wph * np.sin(th) * np.cos(th) * psi
    return out


def _general_directions():
    v = [np.array(x, dtype=float) for x in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    inside = np.array([0.8, 0.35, 0.2])
    edge = v[0] + 0.3 * (v[1] - v[0])                 # on the great circle x-y
    mid = v[0] + v[1]                                  # a level-1 vertex: six patches
    mid2 = (v[0] + v[1]) / np.sqrt(2) + (v[0] + v[2]) / np.sqrt(2)   # a level-2 vertex
    return [("inside", inside), ("edge", edge), ("vertex1", mid), ("vertex2", mid2)]


@pytest.mark.parametrize("basis,paths", MESHES[1:], ids=["lin2", "const1", "aniso3x"])
@pytest.mark.parametrize("name,e", _general_directions(), ids=lambda x: x if isinstance(x, str) else "")
def test_general_beam_weights_are_the_limit_of_a_shrinking_cap(basis, paths, name, e):
    """The share of each patch is the part of a shrinking cap around the beam
    direction that lies in it: inside a patch, on an edge, and at vertices
    where the patches' angles differ (Richardson-extrapolated cap limit)."""
    am = angular.AngularMesh(paths, basis)
    e = e / np.linalg.norm(e)
    wb = transport.beam_weights(am, e)
    f1 = _cap_term_general(am, e, 8e-4)
    f2 = _cap_term_general(am, e, 4e-4)
    assert np.abs((2 * f2 - f1) - wb).max() < 1e-6
    assert abs(wb.sum() - 1.0) < 1e-12


def _general_beam_problem(dim, nc, level, face, val, ss_frac, basis="lin", N=4, g=0.8):
    C = int(np.prod(nc))
    bnd = [(0, 0.0)] * (2 * dim)
    bnd[face] = (3, tuple(val))
    st = np.full(C, 2.0)
    return W.problem(dim, nc, st, ss_frac * st, N, W.hg_moments(g, N), np.zeros(C), level,
                     basis=basis, boundary=bnd)


@pytest.mark.parametrize("dim,nc,face", [(2, (3, 4), 0), (2, (4, 2), 3), (3, (2, 3, 2), 5)])
def test_general_beam_normal_over_the_whole_face_is_the_normal_beam(dim, nc, face):
    S = 1.3
    n = np.zeros(3)
    n[face // 2] = 2.0 * (face % 2) - 1.0
    p2 = _beam_problem(dim, nc, 1, face, S, 0.5)
    p3 = _general_beam_problem(dim, nc, 1, face, [S, *(-n), -1.0, 2.0, -1.0, 2.0], 0.5)
    f2 = _T(p2).source()
    f3 = _T(p3).source()
    assert np.abs(f3 - f2).max() < 1e-14 * np.abs(f2).max()


@pytest.mark.parametrize("dim,nc,face,rng", [
    (2, (5, 7), 0, (0.23, 0.61, 0.0, 0.0)), (2, (6, 4), 2, (0.1, 0.95, 0.0, 0.0)),
    (3, (4, 5, 3), 4, (0.3, 0.7, 0.15, 0.52))])
def test_general_beam_source_total_is_its_incident_current(dim, nc, face, rng):
    """Sum of the source = S |Omega_b.n| |face & range|: the basis functions
    and the patch shares are partitions of unity; the range cuts cells."""
    S = 0.9
    n = np.zeros(3)
    n[face // 2] = 2.0 * (face % 2) - 1.0
    om = -n + np.array([0.3, -0.2, 0.25])
    om /= np.linalg.norm(om)
    p = _general_beam_problem(dim, nc, 1, face, [S, *om, *rng], 0.5)
    f = _T(p).source()
    area = (rng[1] - rng[0]) * ((rng[3] - rng[2]) if dim == 3 else 1.0)
    assert abs(f.sum() - S * abs(om @ n) * area) < 1e-13
    assert (f >= -1e-15).all()


def test_partial_face_beam_solution_balances_and_is_symmetric():
    """3D cube, beam along +z on the square 0.375 < x, y < 0.625 of the low-z
    face (the set-up of Sec. 5.4's cube): the solved flux balances the incident
    current and is symmetric under x <-> y and under x -> 1 - x."""
    nc = (4, 4, 3)
    p = _general_beam_problem(3, nc, 1, 4, [1.0, 0.0, 0.0, 1.0, 0.375, 0.625, 0.375, 0.625],
                              0.7)
    T = _T(p)
    x, _, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 400)
    assert rel < 1e-13
    leak, absn = _leak_and_absorption(T, x)
    assert abs(leak + absn - 0.25 ** 2) < 1e-11
    avg = (T.scalar_flux(x).reshape(T.C, T.s) @ T.cell.mu).reshape(3, 4, 4)   # [z, y, x]
    assert np.abs(avg - avg.transpose(0, 2, 1)).max() < 1e-11 * np.abs(avg).max()
    assert np.abs(avg - avg[:, :, ::-1]).max() < 1e-11 * np.abs(avg).max()
