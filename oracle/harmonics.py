"""Real orthonormal spherical harmonics for the flux-moment form of the
Legendre scatter source (Sec. 4.2, equations for Q, Phi_{n,o} and X).

Oracle (test infrastructure only).

Convention: polar axis z, index k = n*n + n + o for o = -n..n,
    Y_{n,0}  = K(n,0) P_n(z)
    Y_{n,o}  = sqrt(2) K(n,o) P_n^o(z) cos(o*phi)        (o > 0)
    Y_{n,-o} = sqrt(2) K(n,o) P_n^o(z) sin(o*phi)        (o > 0)
with K(n,m)^2 = (2n+1)/(4 pi) (n-m)!/(n+m)! and P_n^m without the
Condon-Shortley phase.  They are orthonormal on the unit sphere, so that
sum_o Y_{n,o}(a) Y_{n,o}(b) = (2n+1)/(4 pi) P_n(a.b) (addition theorem); the
scatter source only ever uses that sum, so the sign/axis convention does not
reach any operator.
"""
import numpy as np


def nmoments(N):
    """Number of real harmonics of degree <= N."""
    return (N + 1) * (N + 1)


def degree_of_index(N):
    """Array deg[k] = n for k = n*n + n + o."""
    deg = np.empty(nmoments(N), dtype=np.int64)
    for n in range(N + 1):
        deg[n * n:(n + 1) * (n + 1)] = n
    return deg


def real_sph_harm(N, omega):
    """Y[..., k] for unit vectors omega[..., 3], all degrees n <= N.

    Normalised associated Legendre functions pbar(n,m) = K(n,m) P_n^m(z) are
    built with the standard three-term recurrence in n at fixed m, started
    from the sectoral values pbar(m,m).
    """
    omega = np.asarray(omega, dtype=np.float64)
    x, y, z = omega[..., 0], omega[..., 1], omega[..., 2]
    sint = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = np.arctan2(y, x)
    shape = omega.shape[:-1]
    Y = np.zeros(shape + (nmoments(N),), dtype=np.float64)

    pmm = np.full(shape, 1.0 / np.sqrt(4.0 * np.pi))
    for m in range(0, N + 1):
        if m > 0:
            pmm = pmm * np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * sint
        # column of pbar(n, m) for n = m..N
        p_nm2 = np.zeros(shape)
        p_nm1 = pmm
        for n in range(m, N + 1):
            if n == m:
                p = pmm
            elif n == m + 1:
                p = np.sqrt(2.0 * m + 3.0) * z * pmm
            else:
                a = np.sqrt((4.0 * n * n - 1.0) / (n * n - m * m))
                b = np.sqrt(((n - 1.0) ** 2 - m * m) / (4.0 * (n - 1.0) ** 2 - 1.0))
                p = a * (z * p_nm1 - b * p_nm2)
            if n > m:
                p_nm2, p_nm1 = p_nm1, p
            base = n * n + n
            if m == 0:
                Y[..., base] = p
            else:
                Y[..., base + m] = np.sqrt(2.0) * p * np.cos(m * phi)
                Y[..., base - m] = np.sqrt(2.0) * p * np.sin(m * phi)
    return Y
