"""Bond lists of the lattices used by the workloads.

Site numbering: site(x, y) = x + Lx * y.  Every geometric bond is emitted once,
also on periodic directions of width 2, where the wrap-around bond coincides
with the direct one (the paper's 2x2 Wannier90 example, Sec. 5, lists such
bonds twice through its hopping file; a caller who wants that doubled value
lists the bond twice).
"""
from __future__ import annotations

MASK64 = (1 << 64) - 1


def _add(bonds: list, seen: set, i: int, j: int) -> None:
    if i == j:
        return
    key = (min(i, j), max(i, j))
    if key in seen:
        return
    seen.add(key)
    bonds.append((i, j))


def chain(L: int, pbc: bool = True) -> list[tuple[int, int]]:
    """Nearest-neighbour bonds (i, i+1) of an L-site chain (Sec. 3.1.1 example)."""
    bonds, seen = [], set()
    for i in range(L - 1 + (1 if pbc else 0)):
        _add(bonds, seen, i, (i + 1) % L)
    return bonds


def square(Lx: int, Ly: int, pbc: bool = True) -> list[tuple[int, int]]:
    """Nearest-neighbour bonds of an Lx x Ly square lattice, site = x + Lx*y."""
    bonds, seen = [], set()
    for y in range(Ly):
        for x in range(Lx):
            s = x + Lx * y
            if x + 1 < Lx or pbc:
                _add(bonds, seen, s, (x + 1) % Lx + Lx * y)
            if y + 1 < Ly or pbc:
                _add(bonds, seen, s, x + Lx * ((y + 1) % Ly))
    return bonds


def ladder(L: int, pbc: bool = True) -> list[tuple[int, int]]:
    """Two-leg ladder of length L: legs along x (periodic), one rung per column."""
    return square(L, 2, pbc=pbc)


def splitmix64_stream(seed: int):
    """SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): yields 64-bit integers."""
    state = seed & MASK64
    while True:
        state = (state + 0x9E3779B97F4A7C15) & MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        yield z ^ (z >> 31)


def random_regular_graph(N: int, degree: int, seed: int, max_tries: int = 100000) -> list[tuple[int, int]]:
    """Random d-regular simple graph by configuration-model pairing with rejection.

    N*degree stubs are shuffled (Fisher-Yates driven by SplitMix64) and paired
    consecutively; a pairing with a self-loop or a repeated edge is rejected and
    the stream continues with a fresh shuffle.
    """
    if (N * degree) % 2:
        raise ValueError("N*degree must be even")
    rng = splitmix64_stream(seed)
    for _ in range(max_tries):
        stubs = [v for v in range(N) for _ in range(degree)]
        for k in range(len(stubs) - 1, 0, -1):
            r = next(rng) % (k + 1)
            stubs[k], stubs[r] = stubs[r], stubs[k]
        edges, seen, ok = [], set(), True
        for a, b in zip(stubs[0::2], stubs[1::2]):
            key = (min(a, b), max(a, b))
            if a == b or key in seen:
                ok = False
                break
            seen.add(key)
            edges.append(key)
        if ok:
            return sorted(edges)
    raise RuntimeError("no simple pairing found")


def uniform_couplings(n: int, lo: float, hi: float, seed: int) -> list[float]:
    """n couplings uniform in [lo, hi): 53-bit uniforms from SplitMix64."""
    rng = splitmix64_stream(seed)
    return [lo + (hi - lo) * ((next(rng) >> 11) * 2.0 ** -53) for _ in range(n)]
