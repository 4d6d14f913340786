"""The allocation-free kernel convolution (vesis_surface_weights_noalloc).

It serves callers that cannot allocate device memory - code inside a CUDA
stream capture, processes whose memory is owned by a pool, loops that must
not enter the allocator - and must give exactly what the system-based
vesis_surface_weights gives.  This file is collected last on purpose, and
it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2208_05524_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n", [(40, 44, 48),      # z in rows of 8: the vector z pass
                               (33, 35, 37),      # nz % 8 != 0: the per-cell z pass
                               (64, 128, 128)])   # exactly VESIS_NOALLOC_MAX_CELLS cells
def test_noalloc_matches_system_path_on_two_calls(n):
    from paper_2208_05524_gb300 import vesis
    h = 0.3
    s = synth.single_ion(n=8, h=h)
    s["n"] = np.array(n)
    s["origin"] = -0.5 * np.array(n) * h
    S = vesis.System(s)
    G = int(np.prod(n))
    assert G <= vesis.NOALLOC_MAX_CELLS
    for call, seed in enumerate((3, 4)):
        chi0 = synth.random_labels(n, seed=seed, p=0.45)
        chi = torch.from_numpy(chi0.reshape(-1)).cuda()
        W_sys = torch.empty(G, dtype=torch.int32, device="cuda")
        S.surface_weights(chi, W_sys)
        W_na = torch.full((G,), -1, dtype=torch.int32, device="cuda")
        vesis.surface_weights_noalloc(S.params, chi, W_na)
        torch.cuda.synchronize()
        # exact integers on both paths
        assert torch.equal(W_na, W_sys), f"call {call}"


def test_noalloc_rejects_oversized_grid():
    from paper_2208_05524_gb300 import vesis
    p = vesis.default_params(nx=128, ny=128, nz=128, h=0.2, origin=(-12.8,) * 3)
    assert p.nx * p.ny * p.nz > vesis.NOALLOC_MAX_CELLS
    chi = torch.zeros(1, dtype=torch.uint8, device="cuda")
    W = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = vesis.lib()
    import ctypes as C
    rc = L.vesis_surface_weights_noalloc(C.byref(p), C.c_void_p(chi.data_ptr()),
                                         C.c_void_p(W.data_ptr()), None)
    assert rc == -1
    assert b"VESIS_NOALLOC_MAX_CELLS" in L.vesis_last_error()
