"""Seeded synthetic inputs for the topology-optimisation solves.

This module only makes inputs (grids, boundary masks, loads, density fields); it contains none
of the method's arithmetic, and both the CUDA path and the CPU oracle consume what it makes.
Layouts follow the library's conventions: 2D node (i, j) -> i + (nx+1) j, 3D node (i, j, k) ->
i + (nx+1)(j + (ny+1) k); DOFs interleaved per node; elements x-fastest.

Workloads (shapes of the paper's Example 2 problems 425/428, Sec. 7.2, and their 3D analogues):
  * ``cantilever_2d``: left edge clamped, unit downward point load at the right-edge midpoint,
    uniform initial density V/m.
  * ``random_field_2d`` / ``random_field_3d``: densities 10^U(-3, 0) smoothed by a normalised
    box filter (mean over the in-bounds cells of a 5-wide window), loads N(0, 1) on the free
    DOFs or unit point loads, x = 0 face clamped.
"""
import numpy as np


def n_dofs(nx, ny, nz=0):
    if nz:
        return 3 * (nx + 1) * (ny + 1) * (nz + 1)
    return 2 * (nx + 1) * (ny + 1)


def clamp_xmin(nx, ny, nz=0):
    """Fixed-DOF mask (uint8, one byte per DOF): every DOF of the nodes with i == 0."""
    d = 3 if nz else 2
    if nz:
        mask = np.zeros((nz + 1, ny + 1, nx + 1, d), dtype=np.uint8)
        mask[:, :, 0, :] = 1
    else:
        mask = np.zeros((ny + 1, nx + 1, d), dtype=np.uint8)
        mask[:, 0, :] = 1
    return mask.reshape(-1)


def point_load(nx, ny, nz, node, comp, value=-1.0):
    """Load vector with a single entry ``value`` on DOF ``comp`` of node (i, j[, k])."""
    d = 3 if nz else 2
    f = np.zeros(n_dofs(nx, ny, nz))
    if nz:
        i, j, k = node
        nid = i + (nx + 1) * (j + (ny + 1) * k)
    else:
        i, j = node
        nid = i + (nx + 1) * j
    f[d * nid + comp] = value
    return f


def box_filter(field, width=5):
    """Mean over the in-bounds cells of a width^dim window centred on each cell."""
    a = np.asarray(field, dtype=float)
    h = width // 2
    out = a
    for axis in range(a.ndim):
        n = a.shape[axis]
        c = np.cumsum(np.moveaxis(out, axis, 0), axis=0)
        c = np.concatenate([np.zeros((1,) + c.shape[1:]), c], axis=0)
        idx = np.arange(n)
        lo = np.clip(idx - h, 0, n)
        hi = np.clip(idx + h + 1, 0, n)
        s = (c[hi] - c[lo])
        out = np.moveaxis(s, 0, axis)
    ones = np.ones_like(a)
    cnt = ones
    for axis in range(a.ndim):
        n = a.shape[axis]
        c = np.cumsum(np.moveaxis(cnt, axis, 0), axis=0)
        c = np.concatenate([np.zeros((1,) + c.shape[1:]), c], axis=0)
        idx = np.arange(n)
        s = c[np.clip(idx + h + 1, 0, n)] - c[np.clip(idx - h, 0, n)]
        cnt = np.moveaxis(s, 0, axis)
    return out / cnt


def log_uniform_field(shape, seed, lo_exp=-3.0, hi_exp=0.0, width=5):
    """Box-filtered 10^U(lo_exp, hi_exp) field (numpy PCG64 with the given seed), values in
    [10^lo_exp, 10^hi_exp]; shape is (ny, nx) or (nz, ny, nx) (x fastest when flattened)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    raw = 10.0 ** rng.uniform(lo_exp, hi_exp, size=shape)
    return box_filter(raw, width).reshape(-1)


def uniform_field(m, seed, lo=1e-3, hi=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=m)


def normal_load(fixed, seed):
    """i.i.d. N(0, 1) entries on the free DOFs, zero on the fixed ones."""
    rng = np.random.Generator(np.random.PCG64(seed))
    f = rng.standard_normal(fixed.shape[0])
    f[np.asarray(fixed, dtype=bool)] = 0.0
    return f


def cantilever_2d(nx, ny, volfrac):
    """Example-2-shaped cantilever: clamp x = 0, f_y = -1 at node (nx, ny/2), V = volfrac * m,
    xbar = 1, x0 = V/m."""
    m = nx * ny
    V = volfrac * m
    return dict(nx=nx, ny=ny, nz=0, fixed=clamp_xmin(nx, ny),
                f=point_load(nx, ny, 0, (nx, ny // 2), 1, -1.0),
                V=V, xbar=1.0, x0=np.full(m, V / m))


def corner_supported_2d(nx, ny, volfrac):
    """Example-3-shaped beam: both components fixed at the two lower corner nodes (0, 0) and
    (nx, 0), f_y = -1 at the lower edge's middle node (nx/2, 0), V = volfrac * m, xbar = 1,
    x0 = V/m."""
    m = nx * ny
    V = volfrac * m
    fixed = np.zeros(n_dofs(nx, ny), dtype=np.uint8)
    for node in (0, nx):
        fixed[2 * node] = fixed[2 * node + 1] = 1
    return dict(nx=nx, ny=ny, nz=0, fixed=fixed, f=point_load(nx, ny, 0, (nx // 2, 0), 1, -1.0),
                V=V, xbar=1.0, x0=np.full(m, V / m))


def random_field_2d(nx, ny, seed_x=0, seed_f=1):
    """Standalone-solve workload: log-uniform smoothed densities, N(0,1) load on free DOFs."""
    fixed = clamp_xmin(nx, ny)
    x = log_uniform_field((ny, nx), seed_x)
    return dict(nx=nx, ny=ny, nz=0, fixed=fixed, f=normal_load(fixed, seed_f), x=x)


def random_field_3d(nx, ny, nz, n_rhs=8, seed_x=2, seed_f=3):
    """3D workload: smoothed log-uniform densities, ``n_rhs`` unit -z point loads at nodes drawn
    uniformly on the x = nx face, x = 0 face clamped.  f is (n_rhs, n)."""
    fixed = clamp_xmin(nx, ny, nz)
    x = log_uniform_field((nz, ny, nx), seed_x)
    rng = np.random.Generator(np.random.PCG64(seed_f))
    F = np.zeros((n_rhs, n_dofs(nx, ny, nz)))
    for r in range(n_rhs):
        j = int(rng.integers(0, ny + 1))
        k = int(rng.integers(0, nz + 1))
        F[r] = point_load(nx, ny, nz, (nx, j, k), 2, -1.0)
    return dict(nx=nx, ny=ny, nz=nz, fixed=fixed, f=F, x=x)


def random_density_problem(nx, ny, nz=0, seed_x=4):
    """Differentiation workload: x ~ U[1e-3, 1]; 2D cantilever load, or in 3D a unit -z load at
    the centre node of the x = nx face."""
    m = nx * ny * (nz if nz else 1)
    x = uniform_field(m, seed_x)
    fixed = clamp_xmin(nx, ny, nz)
    if nz:
        f = point_load(nx, ny, nz, (nx, ny // 2, nz // 2), 2, -1.0)
    else:
        f = point_load(nx, ny, 0, (nx, ny // 2), 1, -1.0)
    return dict(nx=nx, ny=ny, nz=nz, fixed=fixed, f=f, x=x)


def random_vector(n, seed, fixed=None):
    """N(0, 1) vector (zero on fixed DOFs if a mask is given)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal(n)
    if fixed is not None:
        v[np.asarray(fixed, dtype=bool)] = 0.0
    return v
