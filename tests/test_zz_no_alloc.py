"""topo_compliance_noalloc (static device scratch, no allocation) against topo_compliance (the
solver's scratch) on the same seeded vectors, bit for bit, twice in a row so that the ticket counters of the
static scratch are seen to return to zero.  The file name puts it last in collection order, so it
also runs after every other GPU test has used the library."""
import ctypes

import numpy as np
import pytest

from paper_1606_06201_gb300 import workloads as W

from gpu_helpers import dev, host, topo_lib, torch_cuda

pytestmark = pytest.mark.gpu

# (nx, ny, nz, levels, nrhs): a vector shorter than one block, a batch spread over a partial
# reduction grid, a 3D batch, the largest batch the static scratch holds and vectors long enough
# for the full grid of reduction blocks
CASES = [(4, 2, 0, 1, 1), (64, 32, 0, 3, 3), (8, 4, 4, 2, 2), (128, 64, 0, 3, 64),
         (512, 256, 0, 6, 2)]


@pytest.mark.parametrize("nx,ny,nz,levels,nrhs", CASES)
def test_noalloc_matches_solver_compliance_twice(nx, ny, nz, levels, nrhs):
    torch = torch_cuda()
    topo = topo_lib()
    cfg = W.random_density_problem(nx, ny, nz, seed_x=11)
    s = topo.Solver(nx, ny, nz, fixed=cfg["fixed"], levels=levels, nrhs=nrhs)
    rng = np.random.default_rng(12)
    f = dev(torch, rng.standard_normal((nrhs, s.n)))
    u = dev(torch, rng.standard_normal((nrhs, s.n)))
    ref = np.asarray(s.compliance(f, u), dtype=np.float64)
    for _ in range(2):
        c = torch.full((nrhs,), float("nan"), dtype=torch.float64, device="cuda")
        topo.compliance_noalloc(f, u, c, nrhs=nrhs)
        torch.cuda.synchronize()
        got = host(c)
        # the same kernel on the same fixed grid of reduction blocks: the same bits
        scale = np.sqrt(host((f * f).sum(1)) * host((u * u).sum(1)))
        assert np.all(np.abs(got - ref) <= 1e-14 * scale), (got, ref)
        assert np.array_equal(got, ref), (got - ref)
    s.close()


def test_noalloc_empty_and_rejected_sizes():
    torch = torch_cuda()
    topo = topo_lib()
    c = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    e = torch.empty((2, 0), dtype=torch.float64, device="cuda")
    topo.compliance_noalloc(e, e, c, nrhs=2)
    torch.cuda.synchronize()
    assert np.all(host(c) == 0.0)
    v = torch.zeros((65, 8), dtype=torch.float64, device="cuda")
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(topo.TopoError, match="nrhs = 65"):
        topo.compliance_noalloc(v, v, out, nrhs=65)
    lib = topo._lib
    st = lib.topo_compliance_noalloc(None, None, ctypes.c_longlong(-1), 1,
                                     ctypes.c_void_p(out.data_ptr()), None)
    assert st == topo.E_INVALID_ARG
