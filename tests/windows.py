"""Windows of a cube for one-step checks at sizes the oracle cannot run whole (test helper).

One step of a cell reads only its neighbours one cell away (interface reconstruction with
tangential cross points); the wall ghosts and x_c of a true wall lie inside a window that
touches that wall. A window of the state, stepped once by the oracle with the cube's own faces
where it touches them and an artificial rest wall or a periodic seam elsewhere, therefore
gives the exact next state of every window cell at least one cell from an artificial side;
MARGIN = 3 leaves room to spare (pinned in test_windows.py)."""
from paper_1411_6121_gb300 import workloads as W

MARGIN = 3


def window_bcs(lo, win, n, true_bcs):
    """Faces of the window [lo, lo + win) per axis of an n-cell cube with faces true_bcs."""
    bcs = []
    for a in range(3):
        if lo[a] == 0:
            bcs += [true_bcs[2 * a], W.wall()]
        elif lo[a] + win == n:
            bcs += [W.wall(), true_bcs[2 * a + 1]]
        else:
            bcs += [W.periodic(), W.periodic()]
    return bcs


def compared(lo, win, n):
    """Per axis (x, y, z), the window cells whose next state is exact."""
    sl = []
    for a in range(3):
        if lo[a] == 0:
            sl.append(slice(0, win - MARGIN))
        elif lo[a] + win == n:
            sl.append(slice(MARGIN, win))
        else:
            sl.append(slice(MARGIN, win - MARGIN))
    return sl


def starts(n, win, rng, extra=2):
    """Window origins (x, y, z): corners, the lid face, an x wall, an edge, the centre, and
    `extra` random interior ones."""
    e = n - win
    out = [(0, 0, 0), (e, e, e), (0, e, 0), (e, 0, e), (e // 2, e, e // 2), (0, e // 3, e // 2),
           (e // 3, 0, e), (e // 2, e // 2, e // 2)]
    out += [tuple(int(v) for v in rng.integers(1, e, 3)) for _ in range(extra)]
    return out
