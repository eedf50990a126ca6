"""Independent brute-force enumerator of one step's successor distribution.

Test infrastructure, written separately from the C oracle: it states the
probabilistic semantics of one synchronous step (Sec. III, Sec. IV.b-d of
Dutta, McLeod, Friesen) and enumerates them exactly, so that the oracle's
sampled successors can be checked for membership and, for a few agents, for
their frequencies.

Semantics enumerated:
  * an agent on its goal edge column stays;
  * forward cell empty and in the grid -> forward with probability 1;
  * otherwise LEM: the available neighbours ranked by distance to the point
    two cells ahead (ties within the pairs {2,3}, {4,5}, {7,8} in either
    order, each with probability 1/2), rank k drawn from the 12-uniform sum
    rounded half up after clamping at zero, clamped to m-1;
  * ACO: roulette with weights tau*eta over the available neighbours 2..8
    (LEM when every weight is zero);
  * every empty cell with k >= 1 claimants takes one of them uniformly.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np

# agent-frame neighbour i -> (forward component, left-right component); the
# absolute offset for heading s is (s*fx, s*fy) with "left" = -s in y.
FRAME = {1: (1, 0), 2: (1, -1), 3: (1, 1), 4: (0, -1), 5: (0, 1), 6: (-1, 0),
         7: (-1, -1), 8: (-1, 1)}
DIST2 = {i: (2 - fx) ** 2 + fy ** 2 for i, (fx, fy) in FRAME.items()}

U16 = 65536
N12 = 12
MEAN12 = N12 * (U16 - 1) // 2  # 12 * 32767.5 = 393210


def ih12_count_le(T: int) -> int:
    """Number of 12-tuples of integers in [0, 65535] whose sum is <= T
    (inclusion-exclusion over the upper bounds)."""
    if T < 0:
        return 0
    total = 0
    for j in range(N12 + 1):
        r = T - U16 * j
        if r < 0:
            break
        total += (-1) ** j * math.comb(N12, j) * math.comb(r + N12, N12)
    return total


def rank_threshold(j: int, sigma_pow2: int = 0) -> int:
    """Smallest 12-word sum whose rank is >= j (j >= 1) for sigma = 2**p:
    z = (s - mean) * 2^-(16+p) >= j - 1/2."""
    scale = U16 << sigma_pow2
    # s - MEAN12 >= (j - 1/2) * scale, both sides integers when scale even
    return MEAN12 + (2 * j - 1) * scale // 2


def rank_probs(m: int) -> list[Fraction]:
    """Exact probabilities of rank 0..m-1 for sigma = 1."""
    total = U16 ** N12

    def p_ge(j):
        if j <= 0:
            return Fraction(1)
        T = rank_threshold(j)
        return Fraction(total - ih12_count_le(T - 1), total)

    probs = [p_ge(k) - p_ge(k + 1) for k in range(m - 1)]
    probs.append(p_ge(m - 1))
    return probs


_RANK_CACHE: dict[int, list[Fraction]] = {}


def _rank_probs_cached(m):
    if m not in _RANK_CACHE:
        _RANK_CACHE[m] = rank_probs(m)
    return _RANK_CACHE[m]


def eta(i: int) -> float:
    return float(np.float32(1.0 / math.sqrt(DIST2[i])))


def target_distribution(occ, x, y, model=0, tau=None):
    """{frame index: probability} of one agent's proposal (0 = stay)."""
    H, W = occ.shape
    g = int(occ[y, x])
    s = 1 if g == 1 else -1
    if (g == 1 and x == W - 1) or (g == 2 and x == 0):
        return {0: 1.0}

    def free(i):
        fx, fy = FRAME[i]
        nx, ny = x + s * fx, y + s * fy
        return 0 <= nx < W and 0 <= ny < H and occ[ny, nx] == 0

    avail = {i: free(i) for i in FRAME}
    if avail[1]:
        return {1: 1.0}
    if model == 1:
        w = {}
        for i in range(2, 9):
            if avail[i]:
                fx, fy = FRAME[i]
                w[i] = float(np.float32(tau[g - 1][y + s * fy, x + s * fx])) * eta(i)
        S = sum(w.values())
        if S > 0:
            return {i: wi / S for i, wi in w.items() if wi > 0}
    out: dict[int, float] = {}
    for bits in range(8):
        order = [1, 2, 3, 4, 5, 6, 7, 8]
        if bits & 1:
            order[1], order[2] = 3, 2
        if bits & 2:
            order[3], order[4] = 5, 4
        if bits & 4:
            order[6], order[7] = 8, 7
        L = [i for i in order if avail[i]]
        if not L:
            out[0] = out.get(0, 0.0) + 1 / 8
            continue
        pr = _rank_probs_cached(len(L))
        for k, i in enumerate(L):
            if pr[k] > 0:
                out[i] = out.get(i, 0.0) + float(pr[k]) / 8
    return out


def absolute_target(occ, x, y, i):
    g = int(occ[y, x])
    s = 1 if g == 1 else -1
    if i == 0:
        return (x, y)
    fx, fy = FRAME[i]
    return (x + s * fx, y + s * fy)


def legal_targets(occ, x, y, model=0, tau=None):
    """Set of absolute cells the agent at (x, y) proposes with nonzero probability."""
    return {absolute_target(occ, x, y, i) for i in target_distribution(occ, x, y, model, tau)}


def successor_distribution(occ, ids, model=0, tau=None):
    """Exact distribution over successor (occ, ids) states, keyed by bytes."""
    H, W = occ.shape
    agents = [(x, y) for y in range(H) for x in range(W) if occ[y, x]]
    dists = [target_distribution(occ, x, y, model, tau) for (x, y) in agents]
    result: dict[bytes, float] = {}
    for combo in itertools.product(*[list(d.items()) for d in dists]):
        p = 1.0
        targets = {}
        for (x, y), (i, pi) in zip(agents, combo):
            p *= pi
            t = absolute_target(occ, x, y, i)
            if t != (x, y):
                targets.setdefault(t, []).append((x, y))
        cells = sorted(targets)
        choices = [targets[c] for c in cells]
        n_ways = 1
        for ch in choices:
            n_ways *= len(ch)
        for winners in itertools.product(*choices):
            o2 = occ.copy()
            i2 = ids.copy()
            for (tx, ty), (wx, wy) in zip(cells, winners):
                o2[ty, tx] = occ[wy, wx]
                i2[ty, tx] = ids[wy, wx]
                o2[wy, wx] = 0
                i2[wy, wx] = 0
            key = o2.tobytes() + i2.tobytes()
            result[key] = result.get(key, 0.0) + p / n_ways
    return result


def check_successor(occ, ids, occ1, ids1, model=0, tau=None):
    """Membership checks of one observed successor; returns a list of
    violations (empty when the successor is legal)."""
    H, W = occ.shape
    problems = []
    pos0 = {int(ids[y, x]): (x, y) for y in range(H) for x in range(W) if occ[y, x]}
    pos1 = {int(ids1[y, x]): (x, y) for y in range(H) for x in range(W) if occ1[y, x]}
    if set(pos0) != set(pos1):
        problems.append("agent set changed")
        return problems
    for a, (x, y) in pos0.items():
        x1, y1 = pos1[a]
        if occ1[y1, x1] != occ[y, x]:
            problems.append(f"agent {a} changed group")
        legal = legal_targets(occ, x, y, model, tau)
        if (x1, y1) != (x, y):
            if (x1, y1) not in legal:
                problems.append(f"agent {a} moved to an illegal cell {(x1, y1)} from {(x, y)}")
            if occ[y1, x1] != 0:
                problems.append(f"agent {a} entered a cell occupied at t")
        else:
            if (x, y) not in legal:
                # it must have lost: some legal target now holds another agent
                # that was not there at t
                lost = any(occ1[ty, tx] != 0 and occ[ty, tx] == 0 for (tx, ty) in legal)
                if not lost:
                    problems.append(f"agent {a} stayed without a reason at {(x, y)}")
        if len(legal) == 1:
            (tx, ty), = legal
            if (tx, ty) != (x, y) and occ1[ty, tx] == 0:
                problems.append(f"agent {a}'s only target {(tx, ty)} stayed empty")
    return problems
