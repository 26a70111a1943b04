"""A model of the warp-pipelined 2D sweep's hand-over protocol, run on the CPU
under random interleavings of the warps: warp w owns rows RW w .. RW w + RW - 1
and at step t solves cell t - r of its row r; its first row reads the
previous warp's last-row output for cell t from ring slot t mod R once that
warp's step counter reaches t + RW; a warp writes the slot of cell j only
once the next warp's counter shows it has read cell j - R.  Checked: every
interleaving finishes (no two warps wait on each other), and every read finds
the value written for its own cell, neither stale nor overwritten."""
import numpy as np
import pytest

R = 16  # ring slots, as in the kernel


def simulate(nx, ny, G, seed):
    RW = 32 // G
    nwarp = -(-ny // RW)
    nsteps = nx + RW - 1
    rng = np.random.default_rng(seed)
    prog = [0] * nwarp          # steps completed per warp
    phase = [0] * nwarp         # 0: read (wait on w-1), 1: write (wait on w+1)
    ring = {w: [None] * R for w in range(nwarp)}
    reads = 0
    while True:
        ready = []
        for w in range(nwarp):
            ts = prog[w]
            if ts >= nsteps:
                continue
            if phase[w] == 0:
                if w == 0 or ts >= nx or prog[w - 1] >= ts + RW:
                    ready.append(w)
            else:
                jl = ts - (RW - 1)
                if w + 1 >= nwarp or not (0 <= jl < nx) or jl < R or prog[w + 1] >= jl - R + 1:
                    ready.append(w)
        if not ready:
            break
        w = int(rng.choice(ready))
        ts = prog[w]
        if phase[w] == 0:
            if w > 0 and ts < nx:
                got = ring[w - 1][ts % R]
                assert got == ts, (w, ts, got)  # the value of cell ts, not stale
                reads += 1
            phase[w] = 1
        else:
            jl = ts - (RW - 1)
            if w + 1 < nwarp and 0 <= jl < nx:
                ring[w][jl % R] = jl
            prog[w] = ts + 1
            phase[w] = 0
    return all(p == nsteps for p in prog), reads, nwarp


@pytest.mark.parametrize("G", [2, 4, 8])
@pytest.mark.parametrize("nx,ny", [(5, 21), (37, 29), (70, 24), (128, 128), (3, 128)])
def test_every_interleaving_finishes_with_fresh_values(G, nx, ny):
    for seed in range(6):
        done, reads, nwarp = simulate(nx, ny, G, seed)
        assert done
        assert reads == (nwarp - 1) * nx
