"""DG-Q1 spatial element matrices on an axis-aligned box cell (Sec. 2.3).

Oracle (test infrastructure only).

The cell [0,h_x] x [0,h_y] (x [0,h_z]) carries the tensor-product nodal basis
Phi_i = l_a(x) l_b(y) (l_c(z)), i = a + 2b (+ 4c), l_0(t) = 1 - t/h,
l_1(t) = t/h.  Every matrix is the defining integral evaluated by a tensor
Gauss-Legendre rule that is exact for the polynomial degrees involved:
  N_{li}        = int_V Phi_l Phi_i                     (mass)
  V_{li xi}     = int_V d_xi Phi_l Phi_i                (volume streaming)
  Fown_{f,li}   = int_{face f} Phi_l Phi_i              (outflow / own trace)
  Fnb_{f,li}    = int_{face f} Phi_l Phi_i^{nb}         (neighbour's trace)
  mu_l          = int_V Phi_l,   mf_{f,l} = int_{face f} Phi_l
Face f = 2*xi + side, side 0 = low face (outward normal -e_xi), 1 = high.
"""
import itertools

import numpy as np


def _gauss01(n):
    g, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (g + 1.0), 0.5 * w


class Q1Cell:
    def __init__(self, h):
        self.h = np.asarray(h, dtype=np.float64)
        self.dim = len(self.h)
        self.s = 2 ** self.dim
        d, s = self.dim, self.s
        t, wt = _gauss01(3)
        pts = np.array(list(itertools.product(range(3), repeat=d)))
        X = t[pts] * self.h                      # [np, d] physical points
        W = np.prod(wt[pts], axis=1) * np.prod(self.h)
        phi = self.basis(X)                      # [np, s]
        dphi = self.grad(X)                      # [np, d, s]
        self.N = np.einsum("k,kl,ki->li", W, phi, phi)
        self.V = np.einsum("k,kxl,ki->xli", W, dphi, phi)
        self.mu = W @ phi
        self.Fown = np.zeros((2 * d, s, s))
        self.Fnb = np.zeros((2 * d, s, s))
        self.mf = np.zeros((2 * d, s))
        for xi in range(d):
            others = [e for e in range(d) if e != xi]
            fp = np.array(list(itertools.product(range(3), repeat=d - 1))).reshape(-1, d - 1)
            Wf = np.prod(wt[fp], axis=1) * np.prod(self.h[others]) if d > 1 else np.ones(1)
            for side in range(2):
                Xf = np.zeros((fp.shape[0], d))
                for j, e in enumerate(others):
                    Xf[:, e] = t[fp[:, j]] * self.h[e]
                Xf[:, xi] = side * self.h[xi]
                own = self.basis(Xf)
                # neighbour across this face: same physical point, seen from a
                # cell shifted by +-h_xi
                Xn = Xf.copy()
                Xn[:, xi] = Xf[:, xi] - (1.0 if side == 1 else -1.0) * self.h[xi]
                nb = self.basis(Xn)
                f = 2 * xi + side
                self.Fown[f] = np.einsum("k,kl,ki->li", Wf, own, own)
                self.Fnb[f] = np.einsum("k,kl,ki->li", Wf, own, nb)
                self.mf[f] = Wf @ own

    def face_integral(self, f, a, b):
        """int over the part of face f whose tangential coordinates lie in
        [a_e, b_e] (cell-local, one interval per tangential axis e in
        increasing order, already clipped to [0, h_e]) of Phi_l; [s].  The
        same tensor Gauss rule, mapped onto the sub-rectangle."""
        d, s = self.dim, self.s
        xi, side = divmod(f, 2)
        others = [e for e in range(d) if e != xi]
        t, wt = _gauss01(3)
        fp = np.array(list(itertools.product(range(3), repeat=d - 1))).reshape(-1, d - 1)
        Xf = np.zeros((fp.shape[0], d))
        Wf = np.ones(fp.shape[0])
        for j, e in enumerate(others):
            Xf[:, e] = a[j] + t[fp[:, j]] * (b[j] - a[j])
            Wf = Wf * wt[fp[:, j]] * (b[j] - a[j])
        Xf[:, xi] = side * self.h[xi]
        return Wf @ self.basis(Xf)

    def _l(self, a, t, h):
        return (1.0 - t / h) if a == 0 else (t / h)

    def _dl(self, a, h):
        return (-1.0 / h) if a == 0 else (1.0 / h)

    def basis(self, X):
        X = np.atleast_2d(X)
        out = np.ones((X.shape[0], self.s))
        for i in range(self.s):
            for e in range(self.dim):
                ae = (i >> e) & 1
                out[:, i] *= self._l(ae, X[:, e], self.h[e])
        return out

    def grad(self, X):
        X = np.atleast_2d(X)
        out = np.ones((X.shape[0], self.dim, self.s))
        for i in range(self.s):
            for g in range(self.dim):
                for e in range(self.dim):
                    ae = (i >> e) & 1
                    if e == g:
                        out[:, g, i] *= self._dl(ae, self.h[e])
                    else:
                        out[:, g, i] *= self._l(ae, X[:, e], self.h[e])
        return out
