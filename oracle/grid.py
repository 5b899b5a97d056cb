"""Grid hierarchy: sizes and spacings of the levels.

Sec. 4.1 (MGCNN settings) uses 4 levels for a 31x31 grid and one more level per
doubling; with halving coarsening (Sec. 2.3) and stride-2 unpadded 3x3
restriction, an n = 2^m - 1 interior grid nests as n_{l+1} = (n_l - 1) / 2 down
to a 3x3 coarsest grid, which gives L = log2(n + 1) - 1 levels.
"""
from __future__ import annotations

import math


def num_levels(n: int) -> int:
    """L = log2(n+1) - 1; n must be 2^m - 1 with m >= 2."""
    m = int(round(math.log2(n + 1)))
    if n < 3 or (1 << m) - 1 != n:
        raise ValueError(f"n={n} is not of the form 2^m - 1 with m >= 2")
    return m - 1


def level_sizes(n: int, levels: int | None = None) -> list[int]:
    """Interior sizes n_1 = n, n_{l+1} = (n_l - 1)/2 for the requested number of levels."""
    L = num_levels(n) if levels is None else levels
    sizes = [n]
    for _ in range(L - 1):
        nc = (sizes[-1] - 1) // 2
        if nc < 1:
            raise ValueError("too many levels for this grid")
        sizes.append(nc)
    return sizes


def spacing(n_l: int) -> float:
    """Mesh width of a level with n_l interior nodes per side on the unit square."""
    return 1.0 / (n_l + 1)
