"""Shared set-up for the GPU parity tests: builds oracle-side and CUDA-side objects from the same
seeded inputs."""
import numpy as np
import pytest

from oracle import fe, mg
from paper_1606_06201_gb300 import workloads as W


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def topo_lib():
    torch_cuda()
    from paper_1606_06201_gb300 import topo
    return topo


def grid_of(nx, ny, nz=0):
    return fe.Grid(nx, ny, nz)


def dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def oracle_K_free(nx, ny, nz, x, fixed):
    grid = fe.Grid(nx, ny, nz)
    K0 = fe.element_stiffness(grid.dim)
    free = fe.free_dofs(fixed)
    return fe.assemble(grid, K0, x)[free][:, free].tocsr(), free, grid


def oracle_hierarchy(nx, ny, nz, x, fixed, levels):
    K, free, grid = oracle_K_free(nx, ny, nz, x, fixed)
    return mg.hierarchy(grid, np.asarray(fixed, bool), K, levels), free, grid, K


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
