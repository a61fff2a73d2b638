"""Oracle of the path search across slices (Sec. III-D).  Test
infrastructure: only the tests and the benchmark's CPU baseline use it.

The graph, written out from the definitions of Sec. III-D:
- states are (m, i, j): cell (i, j) on the m-th kept slice;
- cells of adjacent kept slices whose ground elevations are equal are the
  same node; the node cost c^N is the minimum of their c^T;
- a state connects to its 8 neighbours on its slice; entering a node costs
  its c^N plus the Euclidean distance between the two nodes, measured in
  cell units (planar offset of 1 or sqrt 2, elevation change divided by
  r_g); a node whose c^N is c^B (or whose ground is invalid) is not entered;
- a gateway joins (m, i, j) to (m+1, i, j) when the ground is equal and
  c^T(m+1) < c^T(m), and to (m-1, i, j) likewise; it costs nothing (the
  same node).
The optimal cost is found by Dijkstra's algorithm without any heuristic,
over every state, with plain Python loops: meant for maps of a few thousand
cells.  The goal is reached by any state on the goal cell with the goal
slice's ground elevation.
"""
from __future__ import annotations

import heapq
import math

import numpy as np


def node_costs(eG: np.ndarray, cT: np.ndarray, kept: list[int], c_b: float) -> np.ndarray:
    """c^N [M, H, W] (float64): per kept slice and cell, the minimum c^T over
    the adjacent kept slices that share the cell's ground elevation."""
    M = len(kept)
    G = eG[kept].astype(np.float64)
    T = cT[kept].astype(np.float64)
    out = np.full(G.shape, float(c_b))
    H, W = G.shape[1:]
    for i in range(H):
        for j in range(W):
            for m in range(M):
                e = G[m, i, j]
                if not math.isfinite(e):
                    continue
                c = T[m, i, j]
                a = m - 1
                while a >= 0 and G[a, i, j] == e:
                    c = min(c, T[a, i, j])
                    a -= 1
                b = m + 1
                while b < M and G[b, i, j] == e:
                    c = min(c, T[b, i, j])
                    b += 1
                out[m, i, j] = c
    return out


def plan(eG: np.ndarray, cT: np.ndarray, keep, c_b: float, res: float, start, goal):
    """Optimal path cost from start to goal, each (i, j, original slice) on a
    kept slice; +inf when the goal cannot be reached.  Returns (cost, path),
    path a list of (i, j, original slice) from start to goal (one of the
    optimal ones)."""
    N, H, W = eG.shape
    kept = [k for k in range(N) if keep is None or keep[k]]
    M = len(kept)
    G = eG[kept].astype(np.float64)
    T = cT[kept].astype(np.float64)
    CN = node_costs(eG, cT, kept, c_b)
    ms, mg = kept.index(start[2]), kept.index(goal[2])
    s0 = (ms, start[0], start[1])
    goal_cell, goal_e = (goal[0], goal[1]), G[mg, goal[0], goal[1]]
    if not (CN[s0] < c_b) or not (CN[mg, goal[0], goal[1]] < c_b):
        return math.inf, []

    def successors(m, i, j):
        e = G[m, i, j]
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                if di == 0 and dj == 0:
                    continue
                ni, nj = i + di, j + dj
                if not (0 <= ni < H and 0 <= nj < W):
                    continue
                ne = G[m, ni, nj]
                if not math.isfinite(ne) or not (CN[m, ni, nj] < c_b):
                    continue
                dz = (ne - e) / res
                yield (m, ni, nj), CN[m, ni, nj] + math.sqrt(di * di + dj * dj + dz * dz)
        for nm in (m - 1, m + 1):
            if 0 <= nm < M and G[nm, i, j] == e and T[nm, i, j] < T[m, i, j]:
                yield (nm, i, j), 0.0

    dist = {s0: 0.0}
    prev = {s0: None}
    heap = [(0.0, s0)]
    done = set()
    while heap:
        d, s = heapq.heappop(heap)
        if s in done:
            continue
        done.add(s)
        m, i, j = s
        if (i, j) == goal_cell and G[m, i, j] == goal_e:
            path = []
            while s is not None:
                path.append((s[1], s[2], kept[s[0]]))
                s = prev[s]
            return d, path[::-1]
        for t, w in successors(m, i, j):
            nd = d + w
            if t not in dist or nd < dist[t]:
                dist[t] = nd
                prev[t] = s
                heapq.heappush(heap, (nd, t))
    return math.inf, []


def path_cost(eG: np.ndarray, cT: np.ndarray, keep, c_b: float, res: float, path) -> float:
    """Cost of a given state sequence under the same definitions; raises
    ValueError when a step is not an edge of the graph."""
    N = eG.shape[0]
    kept = [k for k in range(N) if keep is None or keep[k]]
    CN = node_costs(eG, cT, kept, c_b)
    total = 0.0
    for (i, j, k), (ni, nj, nk) in zip(path[:-1], path[1:]):
        m, nm = kept.index(k), kept.index(nk)
        e, ne = float(eG[k, i, j]), float(eG[nk, ni, nj])
        if (i, j) == (ni, nj) and abs(nm - m) == 1:
            if not (ne == e and float(cT[nk, i, j]) < float(cT[k, i, j])):
                raise ValueError(f"no gateway from {(i, j, k)} to {(ni, nj, nk)}")
            continue
        if nm != m or max(abs(ni - i), abs(nj - j)) != 1:
            raise ValueError(f"{(i, j, k)} -> {(ni, nj, nk)} is not a move")
        if not math.isfinite(ne) or not (CN[nm, ni, nj] < c_b):
            raise ValueError(f"{(ni, nj, nk)} cannot be entered")
        dz = (ne - e) / res
        total += CN[nm, ni, nj] + math.sqrt((ni - i) ** 2 + (nj - j) ** 2 + dz * dz)
    return total
