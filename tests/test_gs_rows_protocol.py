"""A model of the row-pipelined coarse Gauss-Seidel's hand-over protocol
(2D), run on the CPU under random interleavings of the thread blocks: block
b owns rows b, b + nb, ...; for every sweep, every direction in index order
and every owned row in the direction's upwind row order, it visits the row's
cells in the direction's x order; a cell with an upwind row waits until that
row's face word for (direction, cell) carries the current sweep's tag, and
then writes its own face word with that tag.  Checked: every interleaving
finishes (every wait is on a cell earlier in one global order), and no reader
ever finds its word already rewritten by the next sweep."""
import numpy as np
import pytest


def programme(b, nb, nx, ny, sweeps):
    """The cell sequence of block b: (sweep, direction, x, y)."""
    out = []
    for s in range(sweeps):
        for d in range(4):
            bx, by = (d >> 1) & 1, d & 1
            rows = [r for r in range(ny) if r % nb == b]
            rows.sort(key=lambda r: ny - 1 - r if by else r)
            for r in rows:
                for k in range(nx):
                    out.append((s, d, nx - 1 - k if bx else k, r))
    return out


def simulate(nx, ny, nb, sweeps, seed):
    rng = np.random.default_rng(seed)
    prog = [programme(b, nb, nx, ny, sweeps) for b in range(nb)]
    pos = [0] * nb
    tag = {}  # (direction, x, y) -> sweep of the last write
    while True:
        ready = []
        for b in range(nb):
            if pos[b] >= len(prog[b]):
                continue
            s, d, x, y = prog[b][pos[b]]
            up = y + 1 if d & 1 else y - 1
            if 0 <= up < ny:
                t = tag.get((d, x, up), -1)
                assert t <= s, ("face word rewritten before it was read", (s, d, x, y), t)
                if t < s:
                    continue
            ready.append(b)
        if not ready:
            break
        b = int(rng.choice(ready))
        s, d, x, y = prog[b][pos[b]]
        tag[(d, x, y)] = s
        pos[b] += 1
    return all(pos[b] == len(prog[b]) for b in range(nb))


@pytest.mark.parametrize("nx,ny,nb", [(4, 6, 6), (5, 7, 3), (3, 8, 4), (6, 5, 2), (2, 9, 9)])
def test_every_interleaving_finishes_without_overwrites(nx, ny, nb):
    for seed in range(8):
        assert simulate(nx, ny, nb, 3, seed)
