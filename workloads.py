"""Seeded synthetic inputs shaped like the paper's test problems.

This module is shared by the CUDA path's tests/bench and by the CPU oracle.  It
holds none of the method's arithmetic: it only draws meshes, cross sections,
sources and Legendre moment shapes from seeded generators (NumPy PCG64, base
seed 20104559, one stream per workload) and returns them as plain arrays.

A problem is a dict with keys
  dim            2 or 3
  ncell          (nx, ny[, nz])
  lo, hi         box corners (3 floats each; z ignored in 2D)
  sigma_t        float64[C]  total cross section per cell
  sigma_s        float64[C]  scatter cross section sigma_{s,0} per cell
  N              Legendre order of the scatter expansion
  fmom           float64[N+1] moment shape f_n (sigma_{s,n} = sigma_s * f_n), f_0 = 1,
                 or float64[nmat][N+1], one shape per material of mat_id
  mat_id         optional int[C]: material of each cell (index into fmom's rows)
  q              float64[C]  isotropic volumetric source (scalar emission density)
  boundary       list of 2*dim (kind, value): kind 0 vacuum, 1 isotropic inflow
                 of angular flux `value`, 2 normally incident pencil beam of
                 strength `value` uniform over the face; face f = 2*axis + side
                 (side 1 = high)
  basis          "lin" or "const"
  level          uniform angular level of the finest mesh
  mg             dict(nlevels, Nr (per level, finest first), nu_pre, nu_post,
                 coarse_sweeps)
  tol, restart   GMRES stop tolerance on ||r||/||b|| and restart length
Cells are numbered c = ix + nx*(iy + ny*iz).
"""
import numpy as np

BASE_SEED = 20104559


def _rng(k):
    return np.random.Generator(np.random.PCG64([BASE_SEED, k]))


def hg_moments(g, N):
    """Henyey-Greenstein Legendre moment shape f_n = g^n, n = 0..N."""
    return np.array([g ** n for n in range(N + 1)], dtype=np.float64)


def fp_moments(alpha, N):
    """Fokker-Planck-equivalent Legendre moments (Sec. 2.4): sigma_{s,n} =
    alpha/2 (N(N+1) - n(n+1)), n = 0..N.  Returns (sigma_{s,0}, the shape
    f_n = sigma_{s,n} / sigma_{s,0}); sigma_{s,0} - sigma_{s,n} is alpha/2
    times the eigenvalue n(n+1) of the Laplace-Beltrami operator, so the
    truncated expansion acts like alpha/2 times angular diffusion."""
    s0 = 0.5 * alpha * N * (N + 1)
    sn = np.array([0.5 * alpha * (N * (N + 1) - n * (n + 1)) for n in range(N + 1)])
    return s0, sn / s0


def _central_source(dim, ncell, lo, hi, width, strength=1.0):
    """Unit isotropic source in the centred box of side `width` (cell-aligned
    when the mesh is)."""
    nx, ny = ncell[0], ncell[1]
    nz = ncell[2] if dim == 3 else 1
    q = np.zeros(nx * ny * nz)
    c_lo = [0.5 * (lo[e] + hi[e]) - 0.5 * width for e in range(dim)]
    c_hi = [0.5 * (lo[e] + hi[e]) + 0.5 * width for e in range(dim)]
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                idx = (ix, iy, iz)
                inside = True
                for e in range(dim):
                    h = (hi[e] - lo[e]) / ncell[e]
                    mid = lo[e] + (idx[e] + 0.5) * h
                    inside &= c_lo[e] < mid < c_hi[e]
                if inside:
                    q[ix + nx * (iy + ny * iz)] = strength
    return q


def problem(dim, ncell, sigma_t, sigma_s, N, fmom, q, level, basis="lin",
            boundary=None, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), mg=None,
            tol=1e-8, restart=20, mat_id=None):
    if boundary is None:
        boundary = [(0, 0.0)] * (2 * dim)
    out = dict(dim=dim, ncell=tuple(int(n) for n in ncell), lo=tuple(lo),
               hi=tuple(hi), sigma_t=np.asarray(sigma_t, dtype=np.float64),
               sigma_s=np.asarray(sigma_s, dtype=np.float64), N=int(N),
               fmom=np.asarray(fmom, dtype=np.float64),
               q=np.asarray(q, dtype=np.float64), boundary=list(boundary),
               basis=basis, level=int(level), mg=mg, tol=tol, restart=restart)
    if mat_id is not None:
        out["mat_id"] = np.asarray(mat_id, dtype=np.int32)
    return out


def two_shape_problem(dim, ncell, level, N, seed_k, g=(0.9, 0.4), basis="lin"):
    """Small random problem whose cells carry one of two HG moment shapes
    (g per material), material per cell Bernoulli(0.5) from the seed."""
    prob = random_problem(dim, ncell, level, N, seed_k, basis=basis)
    rng = _rng(2000 + seed_k)
    prob["mat_id"] = rng.integers(0, 2, size=int(np.prod(ncell))).astype(np.int32)
    prob["fmom"] = np.stack([hg_moments(gg, N) for gg in g])
    return prob


def config1_square16(level=1):
    """2D unit square, 16x16 cells, level-1 angular mesh (32 patches), HG
    g = 0.8 at order 8, sigma_t = 1, sigma_s = 0.9, unit source in the centred
    0.25 x 0.25 square, vacuum, tol 1e-8, GMRES(20)."""
    nc = (16, 16)
    C = 256
    q = _central_source(2, nc, (0, 0, 0), (1, 1, 1), 0.25)
    mg = dict(nlevels=2, Nr=[8, 4], nu_pre=1, nu_post=1, coarse_sweeps=10)
    return problem(2, nc, np.ones(C), np.full(C, 0.9), 8, hg_moments(0.8, 8), q,
                   level, mg=mg)


def checkerboard(n, block, seed_k):
    """Material index per cell: Bernoulli(0.5) per block x block tile."""
    rng = _rng(seed_k)
    nb = (n + block - 1) // block
    tiles = rng.integers(0, 2, size=(nb, nb))
    mat = np.empty(n * n, dtype=np.int64)
    for iy in range(n):
        for ix in range(n):
            mat[ix + n * iy] = tiles[iy // block, ix // block]
    return mat


def config2_checkerboard(n=128, level=3, N=16, block=16, nlevels=3, Nr=4):
    """2D unit square, n x n cells, two-material checkerboard of block x block
    tiles (seeded), materials (sigma_t, c) = (1, 0.5) and (10, 0.99), HG
    g = 0.9 at order N, centred unit source of side 0.25, vacuum, angular
    level `level`, `nlevels`-level multigrid with coarse order Nr."""
    mat = checkerboard(n, block, 2)
    st = np.where(mat == 0, 1.0, 10.0)
    ss = np.where(mat == 0, 0.5, 9.9)
    q = _central_source(2, (n, n), (0, 0, 0), (1, 1, 1), 0.25)
    mg = dict(nlevels=nlevels, Nr=[N] + [Nr] * (nlevels - 1), nu_pre=1, nu_post=1,
              coarse_sweeps=10)
    return problem(2, (n, n), st, ss, N, hg_moments(0.9, N), q, level, mg=mg)


def config3_cube(n=32, level=2, N=32):
    """3D unit cube, n^3 cells, per-cell sigma_t ~ lognormal(0, 0.5) (seeded),
    sigma_s = 0.9 sigma_t, HG g = 0.95 at order N, centred unit source of
    side 0.25, vacuum, angular level `level`."""
    rng = _rng(3)
    C = n ** 3
    st = np.exp(rng.normal(0.0, 0.5, size=C))
    ss = 0.9 * st
    q = _central_source(3, (n, n, n), (0, 0, 0), (1, 1, 1), 0.25)
    mg = dict(nlevels=min(3, level + 1), Nr=[N] + [9] * 2, nu_pre=1, nu_post=1,
              coarse_sweeps=10)
    mg["Nr"] = mg["Nr"][:mg["nlevels"]]
    return problem(3, (n, n, n), st, ss, N, hg_moments(0.95, N), q, level, mg=mg)


def config4_batch(nprob=256, nmin=16, nmax=96, seed_k=4):
    """Batch of independent 2D problems of uneven size: n ~ U{nmin..nmax}
    cells per axis on the unit square, angular level ~ U{1..3} (Lin), per-cell
    sigma_t ~ lognormal(0, 0.7), HG g ~ U[0.7, 0.95] at order 2*level + 4,
    scatter ratio per problem ~ U[0.5, 0.95], centred unit source of side
    0.25, vacuum; multigrid down to angular level 1 (the coarse mesh of the
    128x128 workload) with coarse order min(N, 4); a level-1 problem is
    preconditioned by the coarse Gauss-Seidel solve alone."""
    rng = _rng(4000 + seed_k)
    out = []
    for _ in range(nprob):
        n = int(rng.integers(nmin, nmax + 1))
        level = int(rng.integers(1, 4))
        N = 2 * level + 4
        C = n * n
        st = np.exp(rng.normal(0.0, 0.7, size=C))
        ss = st * rng.uniform(0.5, 0.95)
        g = rng.uniform(0.7, 0.95)
        q = _central_source(2, (n, n), (0, 0, 0), (1, 1, 1), 0.25)
        mg = dict(nlevels=level, Nr=[N] + [min(N, 4)] * (level - 1), nu_pre=1, nu_post=1,
                  coarse_sweeps=10)
        out.append(problem(2, (n, n), st, ss, N, hg_moments(g, N), q, level, mg=mg))
    return out


def random_problem(dim, ncell, level, N, seed_k, basis="lin", g=0.8,
                   inflow=None):
    """Small random problem for parity tests: lognormal sigma_t, scatter ratio
    U[0.3, 0.95], random non-negative source; optional isotropic inflow on
    every face."""
    rng = _rng(1000 + seed_k)
    C = int(np.prod(ncell))
    st = np.exp(rng.normal(0.0, 0.7, size=C))
    ss = st * rng.uniform(0.3, 0.95, size=C)
    q = rng.uniform(0.0, 1.0, size=C)
    bnd = None
    if inflow is not None:
        bnd = [(1, inflow)] * (2 * dim)
    return problem(dim, ncell, st, ss, N, hg_moments(g, N), q, level, basis=basis,
                   boundary=bnd)


def random_vector(shape, seed_k, dtype=np.float64):
    """Seeded standard-normal test vector."""
    return _rng(5000 + seed_k).standard_normal(shape).astype(dtype)


def table1_cube(N, level=3, n=30, basis="lin", nlevels=None, Nr=2, coarse_sweeps=30):
    """The paper's preliminary test problem (Sec. 5.1, Table 1): a 5 x 5 x 5 cm
    cube of n^3 cells, uniform isotropic unit source, vacuum on all sides,
    Fokker-Planck-equivalent moments sigma_{s,n} = alpha/2 (N(N+1) - n(n+1))
    with alpha = 1.  Reading: the transport cross section sigma_t - sigma_{s,1}
    = 1 with no absorption, so sigma_t = sigma_{s,0} = N(N+1)/2 and
    sigma_t - sigma_{s,1} = alpha = 1.  Multigrid down to angular level 0 with
    order Nr below the finest level; the paper solves its coarsest level to
    1e-5, here `coarse_sweeps` block Gauss-Seidel sweeps stand in for that."""
    s0, f = fp_moments(1.0, N)
    C = n ** 3
    nl = level + 1 if nlevels is None else nlevels
    mg = dict(nlevels=nl, Nr=[N] + [min(N, Nr)] * (nl - 1), nu_pre=1, nu_post=1,
              coarse_sweeps=coarse_sweeps)
    return problem(3, (n, n, n), np.full(C, s0), np.full(C, s0), N, f, np.ones(C), level,
                   basis=basis, hi=(5.0, 5.0, 5.0), mg=mg)


def config5_beam(n=256, level=4, N=64, nlevels=4, Nr=12, g=0.98):
    """2D unit square, n x n cells, sigma_t = 5, sigma_s = 4.95, HG g at order
    N, a normally incident pencil beam of unit strength over the whole low-x
    edge, vacuum elsewhere, no volumetric source, uniform angular level
    `level`, `nlevels`-level multigrid with scatter order Nr below the finest
    level."""
    C = n * n
    bnd = [(2, 1.0), (0, 0.0), (0, 0.0), (0, 0.0)]
    mg = dict(nlevels=nlevels, Nr=[N] + [min(N, Nr)] * (nlevels - 1), nu_pre=1, nu_post=1,
              coarse_sweeps=10)
    return problem(2, (n, n), np.full(C, 5.0), np.full(C, 4.95), N, hg_moments(g, N),
                   np.zeros(C), level, boundary=bnd, mg=mg)
