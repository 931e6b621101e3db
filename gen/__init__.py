"""Seeded synthetic inputs for the interior-point solver.

This module is shared by the CPU oracle's tests, the CUDA path's tests and the
benchmark. It holds none of the method's arithmetic: it draws random streams
(SplitMix64 -> uniform -> Box-Muller normals), builds problem data for the LP
families and computes fill-reducing orderings, which both solvers take as a
given input (the paper computes the ordering once, on the host, and reuses it:
Sec. 2, "GPU Direct Solvers for Optimization").

Problem form (Sec. 1, problem (1)): min f(x) s.t. g(x) >= 0. The LP families
here are  min c^T x  s.t.  A x >= b,  l <= x <= u.

Orderings are returned as ``perm`` with ``perm[k]`` = original index of the
k-th variable eliminated (new -> old).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014), on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, stream: int) -> int:
    """Independent sub-seed for a named stream of a seed."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GAMMA + np.uint64(stream & 0xFFFFFFFF) * _M2
        return int(_mix(np.array([z], dtype=np.uint64))[0])


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Counter-based SplitMix64: element k is mix(seed + (offset + k + 1) * gamma)."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
    return _mix(z)


def uniform(seed: int, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """U[lo, hi) doubles from the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def normal(seed: int, count: int, mean: float = 0.0, std: float = 1.0) -> np.ndarray:
    """N(mean, std^2) by Box-Muller on pairs of SplitMix64 uniforms (cosine branch)."""
    u = (splitmix64(seed, 2 * count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    return mean + std * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class LP:
    """min c^T x  s.t.  A x >= b,  l <= x <= u  (A is m x n CSR)."""

    n: int
    m: int
    rowptr: np.ndarray  # int64, m+1
    col: np.ndarray     # int32, nnz (ascending within a row)
    val: np.ndarray     # float64, nnz
    b: np.ndarray
    c: np.ndarray
    l: np.ndarray
    u: np.ndarray
    x0: np.ndarray | None = None  # the interior point the data was built around
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def dense_A(self) -> np.ndarray:
        A = np.zeros((self.m, self.n))
        for i in range(self.m):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            A[i, self.col[s:e]] = self.val[s:e]
        return A

    def matvec(self, x: np.ndarray) -> np.ndarray:
        rows = np.repeat(np.arange(self.m), np.diff(self.rowptr))
        return np.bincount(rows, weights=self.val * x[self.col], minlength=self.m)

    def rmatvec(self, y: np.ndarray) -> np.ndarray:
        rows = np.repeat(np.arange(self.m), np.diff(self.rowptr))
        return np.bincount(self.col, weights=self.val * y[rows], minlength=self.n)


def _finish_lp(n, m, rowptr, col, val, seed, lo, hi, name) -> LP:
    """b = A x0 - s0 with x0 ~ U(1,9)-scaled interior, s0 ~ U(0.1,1);
    c = A^T y0 + z0 with y0 ~ U(0,1), z0 ~ U(0.1,1)."""
    span = hi - lo
    x0 = lo + span * uniform(stream_seed(seed, 11), n, 0.1, 0.9)
    s0 = uniform(stream_seed(seed, 12), m, 0.1, 1.0)
    y0 = uniform(stream_seed(seed, 13), m, 0.0, 1.0)
    z0 = uniform(stream_seed(seed, 14), n, 0.1, 1.0)
    lp = LP(n, m, rowptr, col, val, np.zeros(m), np.zeros(n),
            np.full(n, float(lo)), np.full(n, float(hi)), x0=x0, name=name)
    lp.b = lp.matvec(x0) - s0
    lp.c = lp.rmatvec(y0) + z0
    return lp


def random_lp(n: int, m: int, per_row: int = 5, seed: int = 0,
              lo: float = 0.0, hi: float = 10.0) -> LP:
    """Random sparse LP: each row has ``per_row`` distinct uniform-random columns
    with N(0,1) values. With n=2000, m=1000, 5 per row, bounds [0,10] this is the
    small-LP workload (x0 ~ U(1,9) when lo=0, hi=10)."""
    per_row = min(per_row, n)
    cand = 8 * per_row + 8
    draws = splitmix64(stream_seed(seed, 1), m * cand).reshape(m, cand)
    cols = (draws % np.uint64(n)).astype(np.int64)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    col_list = []
    for i in range(m):
        seen = []
        for cnd in cols[i]:
            if cnd not in seen:
                seen.append(int(cnd))
                if len(seen) == per_row:
                    break
        assert len(seen) == per_row, "not enough distinct candidate columns"
        col_list.append(sorted(seen))
        rowptr[i + 1] = rowptr[i] + per_row
    col = np.array([c for r in col_list for c in r], dtype=np.int32)
    val = normal(stream_seed(seed, 2), int(rowptr[-1]))
    return _finish_lp(n, m, rowptr, col, val, seed, lo, hi, f"random_lp_{n}x{m}_s{seed}")


def grid_lp(gx: int, gy: int | None = None, gz: int | None = None, seed: int = 1,
            diag_boost: float = 8.0, lo: float = 0.0, hi: float = 10.0) -> LP:
    """Structured LP on a gx x gy x gz grid: one variable and one row per grid
    point; row i holds the 7-point stencil support of point i (non-periodic: only
    in-grid neighbours), values N(0,1), diagonal + ``diag_boost``. Index of
    (x, y, z) is x + gx*(y + gy*z)."""
    gy = gx if gy is None else gy
    gz = gx if gz is None else gz
    n = gx * gy * gz
    idx = np.arange(n, dtype=np.int64)
    x = idx % gx
    y = (idx // gx) % gy
    z = idx // (gx * gy)
    # neighbour offsets in ascending column order: -z, -y, -x, self, +x, +y, +z
    offs = [(-gx * gy, z > 0), (-gx, y > 0), (-1, x > 0), (0, np.ones(n, bool)),
            (1, x < gx - 1), (gx, y < gy - 1), (gx * gy, z < gz - 1)]
    valid = np.stack([v for _, v in offs], axis=1)
    cols = idx[:, None] + np.array([o for o, _ in offs], dtype=np.int64)[None, :]
    counts = valid.sum(1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = cols[valid].astype(np.int32)
    val = normal(stream_seed(seed, 2), int(rowptr[-1]))
    diag_pos = rowptr[:-1] + (valid[:, :3].sum(1))
    val[diag_pos] += diag_boost
    return _finish_lp(n, n, rowptr, col, val, seed, lo, hi, f"grid_lp_{gx}x{gy}x{gz}_s{seed}")


def nd_order_grid3d(gx: int, gy: int | None = None, gz: int | None = None,
                    leaf: int = 64) -> np.ndarray:
    """Geometric nested dissection of a gx x gy x gz grid whose coupling reaches
    two steps along an axis (the pattern of A^T A for a 7-point A).

    A box with at most ``leaf`` points is numbered in ascending index. Otherwise
    the longest side (ties: x, then y, then z) of length L is cut by the two
    planes at lo + floor((L-2)/2) and the next one; the lower part is numbered
    first, then the upper part, then the separator (ascending index)."""
    gy = gx if gy is None else gy
    gz = gx if gz is None else gz
    out: list[np.ndarray] = []

    def box_ids(b):
        (x0, x1), (y0, y1), (z0, z1) = b
        xs = np.arange(x0, x1)
        ys = np.arange(y0, y1)
        zs = np.arange(z0, z1)
        ids = xs[None, None, :] + gx * (ys[None, :, None] + gy * zs[:, None, None])
        return np.sort(ids.ravel())

    # explicit stack; items are ("box", box) or ("emit", ids)
    stack = [("box", ((0, gx), (0, gy), (0, gz)))]
    while stack:
        kind, item = stack.pop()
        if kind == "emit":
            out.append(item)
            continue
        b = item
        lens = [hi - lo for lo, hi in b]
        vol = lens[0] * lens[1] * lens[2]
        if vol == 0:
            continue
        if vol <= leaf:
            out.append(box_ids(b))
            continue
        d = int(np.argmax(lens))  # first maximum: x before y before z
        lo, hi = b[d]
        p = lo + (lens[d] - 2) // 2
        left = list(b)
        left[d] = (lo, p)
        sep = list(b)
        sep[d] = (p, min(p + 2, hi))
        right = list(b)
        right[d] = (min(p + 2, hi), hi)
        # processed in LIFO order: left, right, then separator
        stack.append(("emit", box_ids(tuple(sep))))
        stack.append(("box", tuple(right)))
        stack.append(("box", tuple(left)))
    perm = np.concatenate(out).astype(np.int32)
    assert perm.size == gx * gy * gz
    return perm


def normal_graph(lp_or_rowptr, col=None, n=None):
    """Adjacency (list of sorted neighbour arrays) of the pattern of J^T J for an
    m x n CSR pattern J. Used only to compute an ordering."""
    if isinstance(lp_or_rowptr, LP):
        rowptr, col, n = lp_or_rowptr.rowptr, lp_or_rowptr.col, lp_or_rowptr.n
    else:
        rowptr = lp_or_rowptr
    nbr = [set() for _ in range(n)]
    for r in range(len(rowptr) - 1):
        cs = col[rowptr[r]:rowptr[r + 1]]
        for a in cs:
            nbr[a].update(int(c) for c in cs if c != a)
    return [np.array(sorted(s), dtype=np.int64) for s in nbr]


def min_degree_order(adj: list[np.ndarray]) -> np.ndarray:
    """Exact minimum degree on the elimination graph (ties -> lowest index).
    Dense boolean adjacency: meant for problems of a few thousand variables."""
    n = len(adj)
    G = np.zeros((n, n), dtype=bool)
    for i, a in enumerate(adj):
        G[i, a] = True
    np.fill_diagonal(G, False)
    alive = np.ones(n, dtype=bool)
    deg = G.sum(1).astype(np.int64)
    perm = np.empty(n, dtype=np.int32)
    big = np.iinfo(np.int64).max
    for k in range(n):
        d = np.where(alive, deg, big)
        v = int(np.argmin(d))
        perm[k] = v
        nb = np.flatnonzero(G[v] & alive)
        alive[v] = False
        G[v, :] = False
        G[:, v] = False
        if nb.size:
            sub = np.ix_(nb, nb)
            G[sub] = True
            G[nb, nb] = False
            deg[nb] = G[nb].sum(1)
    return perm


def lp_ordering(lp: LP, method: str = "auto", grid: tuple[int, int, int] | None = None) -> np.ndarray:
    """Ordering used for an LP: geometric ND for grid problems, exact minimum
    degree for small general patterns, identity otherwise."""
    if grid is not None and method in ("auto", "nd"):
        return nd_order_grid3d(*grid)
    if method in ("auto", "md") and lp.n <= 6000:
        return min_degree_order(normal_graph(lp))
    return np.arange(lp.n, dtype=np.int32)


def sgm10(times, shift: float = 10.0) -> float:
    """Shifted geometric mean (prod(t_i + 10))^(1/n) - 10 used to aggregate
    solve times (Sec. 5, Table 1 caption)."""
    t = np.asarray(times, dtype=np.float64)
    return float(np.exp(np.mean(np.log(t + shift))) - shift)


@dataclass
class MPCBatch:
    """Batch of linear MPC QPs (one per instance), stage k = 0..T-1:

        min 1/2 sum_k (x_{k+1}^T Q x_{k+1} + u_k^T R u_k)
        s.t. x_{k+1} = A_k x_k + B_k u_k  (x_0 given),  |u| <= u_max,  |x| <= x_max.

    Arrays are stacked over instances; instance i owns stages
    stage_off[i] .. stage_off[i] + T[i] - 1 of A (12x12) and B (12x4)."""

    T: np.ndarray          # int32, horizons
    stage_off: np.ndarray  # int64, first stage of each instance
    A: np.ndarray          # (sum T, nx, nx)
    B: np.ndarray          # (sum T, nx, nu)
    Q: np.ndarray          # (count, nx) diagonal
    R: np.ndarray          # (count, nu) diagonal
    x0: np.ndarray         # (count, nx)
    u_max: float = 1.0
    x_max: float = 5.0

    @property
    def count(self) -> int:
        return len(self.T)

    def instance(self, i: int):
        s0, t = int(self.stage_off[i]), int(self.T[i])
        return (self.A[s0:s0 + t], self.B[s0:s0 + t], self.Q[i], self.R[i], self.x0[i])


def mpc_batch(count: int = 4096, seed: int = 3, t_min: int = 10, t_max: int = 100,
              nx: int = 12, nu: int = 4, rho: float = 0.95, u_max: float = 1.0,
              x_max: float = 5.0) -> MPCBatch:
    """Instance i uses sub-seed (seed, i): T ~ U{t_min..t_max}; A_k = rho G_k /
    spectral_radius(G_k) with G_k ~ N(0,1); B_k ~ N(0,1); Q, R diagonal ~ U(0.1, 10)
    shared by the stages of an instance; x0 ~ U(-1,1), redrawn (next sub-seed
    draw) until the u = 0 trajectory stays within |x| <= x_max."""
    Ts, As, Bs, Qs, Rs, X0 = [], [], [], [], [], []
    for i in range(count):
        si = stream_seed(seed, 1000 + i)
        T = t_min + int(splitmix64(stream_seed(si, 1), 1)[0] % np.uint64(t_max - t_min + 1))
        G = normal(stream_seed(si, 2), T * nx * nx).reshape(T, nx, nx)
        A = np.empty_like(G)
        for k in range(T):
            A[k] = rho * G[k] / np.max(np.abs(np.linalg.eigvals(G[k])))
        B = normal(stream_seed(si, 3), T * nx * nu).reshape(T, nx, nu)
        Q = uniform(stream_seed(si, 4), nx, 0.1, 10.0)
        R = uniform(stream_seed(si, 5), nu, 0.1, 10.0)
        for draw in range(1000):
            x0 = uniform(stream_seed(si, 100 + draw), nx, -1.0, 1.0)
            x, ok = x0.copy(), True
            for k in range(T):
                x = A[k] @ x
                if np.abs(x).max() > x_max:
                    ok = False
                    break
            if ok:
                break
        Ts.append(T); As.append(A); Bs.append(B); Qs.append(Q); Rs.append(R); X0.append(x0)
    T = np.array(Ts, dtype=np.int32)
    off = np.zeros(count, dtype=np.int64)
    off[1:] = np.cumsum(T)[:-1]
    return MPCBatch(T=T, stage_off=off, A=np.concatenate(As), B=np.concatenate(Bs),
                    Q=np.array(Qs), R=np.array(Rs), x0=np.array(X0), u_max=u_max, x_max=x_max)


def mpc_instance_qp(A, B, Q, R, x0, u_max=1.0, x_max=5.0):
    """One MPC instance as  min c^T z + 1/2 z^T W z,  J z >= b,  l <= z <= u  with
    z = (u_0, x_1, u_1, x_2, ...): the dynamics are the row pairs h >= 0, -h >= 0,
    h_k = x_{k+1} - A_k x_k - B_k u_k (x_0 moves to the right-hand side).
    Returns (LP-shaped data, W as lower CSC (diagonal))."""
    T, nx, nu = A.shape[0], A.shape[1], B.shape[2]
    ns = nu + nx
    n = ns * T
    rows, cols, vals, b = [], [], [], []
    for k in range(T):
        for sign in (1.0, -1.0):
            for r in range(nx):
                ent = {}
                if k > 0:
                    for j in range(nx):
                        ent[(k - 1) * ns + nu + j] = -A[k][r, j]
                for j in range(nu):
                    ent[k * ns + j] = ent.get(k * ns + j, 0.0) - B[k][r, j]
                ent[k * ns + nu + r] = ent.get(k * ns + nu + r, 0.0) + 1.0
                rhs = (A[0][r] @ x0) if k == 0 else 0.0
                cs = sorted(ent)
                rows.append(cs)
                vals.append([sign * ent[c] for c in cs])
                b.append(sign * rhs)
    m = len(rows)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([c for r in rows for c in r], dtype=np.int32)
    val = np.array([v for r in vals for v in r])
    lo = np.concatenate([np.r_[np.full(nu, -u_max), np.full(nx, -x_max)] for _ in range(T)])
    wdiag = np.concatenate([np.r_[R, Q] for _ in range(T)])
    lp = LP(n, m, rowptr, col, val, np.array(b), np.zeros(n), lo, -lo, name=f"mpc_T{T}")
    wp = np.arange(n + 1, dtype=np.int64)
    wi = np.arange(n, dtype=np.int32)
    return lp, (wp, wi, wdiag)


# ---------------------------------------------------------------------------
# Grid NLP: min 1/2 ||u - u_t||^2 + alpha/2 ||v||^2  s.t.  -Lap u + c3 u^3 - v = 0
# (as the pair of rows h >= 0, -h >= 0), v_lo <= v <= v_hi, on an N x N grid
# of interior points (spacing 1/(N+1), u = 0 on the boundary).
# ---------------------------------------------------------------------------
@dataclass
class GridNLP:
    N: int
    alpha: float
    v_lo: float
    v_hi: float
    cubic: int           # 1: the u^3 term is present
    v_bounded: int       # 1: v_lo <= v <= v_hi
    ut: np.ndarray       # target, N*N, index ix + N*iy
    rowptr: np.ndarray   # J pattern (2 N^2 rows, CSR, ascending columns)
    col: np.ndarray
    l: np.ndarray
    u: np.ndarray
    wp: np.ndarray       # W pattern: lower CSC, diagonal only
    wi: np.ndarray

    @property
    def n(self) -> int:
        return 2 * self.N * self.N

    @property
    def m(self) -> int:
        return 2 * self.N * self.N


def grid_nlp_pattern(N: int):
    """CSR pattern of the Jacobian of [h; -h]: row of grid point (ix, iy) holds
    u at (iy-1), (ix-1), centre, (ix+1), (iy+1) (those inside the grid, in this
    order = ascending index) and then v of the point; rows N^2.. repeat it."""
    NN = N * N
    rows = []
    for idx in range(NN):
        ix, iy = idx % N, idx // N
        c = []
        if iy > 0: c.append(idx - N)
        if ix > 0: c.append(idx - 1)
        c.append(idx)
        if ix < N - 1: c.append(idx + 1)
        if iy < N - 1: c.append(idx + N)
        c.append(NN + idx)
        rows.append(c)
    rows = rows + rows
    rowptr = np.zeros(len(rows) + 1, np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate([np.asarray(r, np.int32) for r in rows])
    return rowptr, col


def grid_nlp(N: int = 512, seed: int = 5, alpha: float = 5e-3, v_lo: float = -1.0,
             v_hi: float = 1.0, cubic: int = 1, v_bounded: int = 1) -> GridNLP:
    """Target u_t = sin(pi x) sin(pi y) + N(0, 0.01) (standard deviation 0.1)
    at x = (ix + 1) h, y = (iy + 1) h, h = 1 / (N + 1)."""
    NN = N * N
    h = 1.0 / (N + 1)
    ix = np.arange(NN) % N
    iy = np.arange(NN) // N
    ut = np.sin(np.pi * (ix + 1) * h) * np.sin(np.pi * (iy + 1) * h) + normal(seed, NN, 0.0, 0.1)
    rowptr, col = grid_nlp_pattern(N)
    l = np.full(2 * NN, -np.inf)
    u = np.full(2 * NN, np.inf)
    if v_bounded:
        l[NN:] = v_lo
        u[NN:] = v_hi
    wp = np.arange(2 * NN + 1, dtype=np.int64)
    wi = np.arange(2 * NN, dtype=np.int32)
    return GridNLP(N, alpha, v_lo, v_hi, cubic, v_bounded, ut, rowptr, col, l, u, wp, wi)


def nd_order_grid_nlp(N: int, leaf: int = 64) -> np.ndarray:
    """Nested dissection of the N x N grid (coupling reach two steps, as for the
    squared Laplacian), each point contributing u then v."""
    pts = nd_order_grid3d(N, N, 1, leaf=leaf).astype(np.int64)
    out = np.empty(2 * pts.size, np.int32)
    out[0::2] = pts
    out[1::2] = pts + N * N
    return out
