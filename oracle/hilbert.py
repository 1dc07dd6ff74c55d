"""Hilbert curves over integer grids (exact integer arithmetic).

Test infrastructure only (see the package docstring).

* ``listing1_cells(a)``: the visit order of the standard Hilbert curve of
  order a over the 2^a x 2^a grid, defined by Listing 1 (Section 3): a turtle
  that starts left of (0, 0), first steps right onto (0, 0), and then moves by
  unit steps in direction d (0 right, 1 up, 2 left, 3 down, taken mod 4); a
  curve of order k with heading d and turn sense r is: turn by r, draw order
  k-1 with sense -r, step; turn back by r, draw order k-1 with sense r, step,
  draw order k-1 with sense r; turn back by r, step, draw order k-1 with sense
  -r. Written here as an explicit-stack walk, not as the listing's recursion.
* ``textbook_cells(a)``: the classic bit-by-bit index-to-(x, y) conversion of
  the Hilbert curve (as in Warren, Hacker's Delight, ch. 16), an independent
  definition used to pin ``listing1_cells``.
* ``generalized_cells(W, H)``: a Hilbert-like Hamiltonian path over any W x H
  grid. Section 3 cites Cerveny (2020) for curves over rectangles of arbitrary
  side lengths and states that they coincide with the standard curve when the
  sides are powers of two; the paper gives no algorithm. The recursion below
  follows the construction of Cerveny's generalized Hilbert ("gilbert")
  curve: a long block (2w > 3h) is cut in two along its length, otherwise it
  is cut into a transposed lower-left part, the full-width upper part and a
  reversed lower-right part. The parity rules for the cut positions and the
  top-level orientation are written out here (the library implements the
  same statement independently):

  path(O, A, B): cells O + i a + j b for 0 <= i < w = |A|, 0 <= j < h = |B|
  (a, b unit vectors of A, B), starting at O and ending at O + (w-1) a.
    - h == 1: the w cells along a.          - w == 1: the h cells along b.
    - 2w > 3h ("long"): split A at w1 = floor(w/2), made even when h is even
      and w1 > 1 (w1 -= 1 if odd); path(O, w1 a, B); path(O + w1 a, (w-w1) a, B).
    - otherwise: h1 = floor(h/2), incremented when odd and h > 2;
      w1 = floor(w/2);
        path(O, h1 b, w1 a)                                  (lower-left, transposed)
        path(O + h1 b, A, (h-h1) b)                           (upper part)
        path(O + (w-1) a + (h1-1) b, -h1 b, -(w-w1) a)        (lower-right, reversed)
  Top level: path((0,0), W x, H y) unless W is odd and H even, in which case
  path((0,0), H y, W x) (a unit-step path from (0,0) to (W-1,0) cannot exist
  then, by a checkerboard parity argument). With these parity choices every
  sub-problem admits a unit-step path, so consecutive cells always share an
  edge; for W = H = 2^a the path is the standard curve of Listing 1.
"""
from __future__ import annotations

import numpy as np

_DIRS = ((1, 0), (0, 1), (-1, 0), (0, -1))


def listing1_cells(a: int) -> np.ndarray:
    """(4^a, 2) array of cells in the order Listing 1 visits them."""
    x, y = -1, 0
    out = []

    def move(d):
        nonlocal x, y
        dx, dy = _DIRS[d & 3]
        x += dx
        y += dy
        out.append((x, y))

    move(0)
    # explicit stack of pending actions: ("curve", heading, sense, order) / ("step", heading)
    stack = [("curve", 0, 1, a)]
    while stack:
        item = stack.pop()
        if item[0] == "step":
            move(item[1])
            continue
        _, d, r, k = item
        if k == 0:
            continue
        d1 = d + r            # after the first turn
        d2 = d1 - r           # after turning back
        d3 = d2 - r           # after turning back again
        seq = [("curve", d1, -r, k - 1), ("step", d1),
               ("curve", d2, r, k - 1), ("step", d2),
               ("curve", d2, r, k - 1), ("step", d3),
               ("curve", d3, -r, k - 1)]
        stack.extend(reversed(seq))
    return np.array(out, dtype=np.int64)


def textbook_cells(a: int) -> np.ndarray:
    """Cells of the order-a Hilbert curve by index-to-cell conversion."""
    n = 1 << a
    out = np.zeros((n * n, 2), dtype=np.int64)
    for d in range(n * n):
        x = y = 0
        t = d
        s = 1
        while s < n:
            rx = (t >> 1) & 1
            ry = (t ^ rx) & 1
            if ry == 0:                 # rotate/flip the sub-square
                if rx == 1:
                    x, y = s - 1 - x, s - 1 - y
                x, y = y, x
            x += s * rx
            y += s * ry
            t >>= 2
            s <<= 1
        out[d] = (x, y)
    return out


def _sgn(v):
    return (v > 0) - (v < 0)


def generalized_cells(W: int, H: int) -> np.ndarray:
    """(W*H, 2) cells of the generalized curve stated in the module docstring."""
    if W < 1 or H < 1:
        raise ValueError("grid sides must be positive")
    out = []
    if W % 2 == 1 and H % 2 == 0:
        stack = [(0, 0, 0, H, W, 0)]
    else:
        stack = [(0, 0, W, 0, 0, H)]
    while stack:
        ox, oy, ax, ay, bx, by = stack.pop()
        w = abs(ax) + abs(ay)
        h = abs(bx) + abs(by)
        uax, uay = _sgn(ax), _sgn(ay)
        ubx, uby = _sgn(bx), _sgn(by)
        if h == 1:
            for i in range(w):
                out.append((ox + i * uax, oy + i * uay))
            continue
        if w == 1:
            for j in range(h):
                out.append((ox + j * ubx, oy + j * uby))
            continue
        if 2 * w > 3 * h:
            w1 = w // 2
            if h % 2 == 0 and w1 % 2 == 1 and w1 > 1:
                w1 -= 1
            parts = [(ox, oy, w1 * uax, w1 * uay, bx, by),
                     (ox + w1 * uax, oy + w1 * uay, (w - w1) * uax, (w - w1) * uay, bx, by)]
        else:
            h1 = h // 2
            if h1 % 2 == 1 and h > 2:
                h1 += 1
            w1 = w // 2
            parts = [(ox, oy, h1 * ubx, h1 * uby, w1 * uax, w1 * uay),
                     (ox + h1 * ubx, oy + h1 * uby, ax, ay, (h - h1) * ubx, (h - h1) * uby),
                     (ox + (w - 1) * uax + (h1 - 1) * ubx, oy + (w - 1) * uay + (h1 - 1) * uby,
                      -h1 * ubx, -h1 * uby, -(w - w1) * uax, -(w - w1) * uay)]
        stack.extend(reversed(parts))
    return np.array(out, dtype=np.int64)


def rank_grid(W: int, H: int) -> np.ndarray:
    """rank[x, y] = position of cell (x, y) along the generalized curve."""
    cells = generalized_cells(W, H)
    rank = np.full((W, H), -1, dtype=np.int64)
    rank[cells[:, 0], cells[:, 1]] = np.arange(cells.shape[0])
    return rank
