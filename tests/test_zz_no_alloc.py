"""The allocation-free synthesis entry point against the context-based one.

Some callers cannot allocate device memory when they need a field (a serving
loop with a fixed memory budget, a host arena that owns all device memory,
code that must not trigger the synchronisation of cudaMalloc/cudaFree).
fh_synthesize_static serves them from a static device array; this test checks
through the C ABI that two calls in a row give the same field as
fh_synthesize, within the parity tolerance.  It sits in its own file, named to
be collected last.
"""
import numpy as np
import pytest

import fh_inputs as fi
from paper_1807_02718_gb300 import fh as F

pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


# (J, n_T): a small mesh; J > 1025 (direct near sums, weights shared memory
# above 48 KB); the largest J; and J * n_T at the scratch limit 2^19, where
# the far table's power table, aliased with the weight planes, is largest.
SIZES = [(96, 360), (1100, 524288 // 1100), (2049, 524288 // 2049)]


@pytest.mark.parametrize("J,n_T", SIZES)
def test_static_scratch_synthesis_matches_context_path(J, n_T):
    import torch
    from paper_1807_02718_gb300 import build
    build.build()
    W = 20.0 * (J - 1) / 95.0
    wl = fi.kite_pulses(J=J, W=W, n_x=40, n_near=n_T - n_T // 6, n_far=n_T // 6)
    assert wl.T.size == n_T
    pr = F.Problem()
    pr.discretize(wl.curve, wl.omega, wl.N)
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    s, B = F.fh_get_window_spectra(pr.ctx, wl.J)
    rng = np.random.default_rng(3)
    V = rng.standard_normal((wl.n_x, wl.J)) + 1j * rng.standard_normal((wl.n_x, wl.J))
    V[:, 0] = 1.0
    u_ref = F.fh_synthesize(pr.ctx, V, wl.T)

    dev = torch.device("cuda", 0)
    d_s = torch.tensor(s, device=dev)
    d_B = torch.tensor(np.ascontiguousarray(B).view(np.float64).ravel(), device=dev)
    d_V = torch.tensor(np.ascontiguousarray(V.T).view(np.float64).ravel(), device=dev)
    d_T = torch.tensor(wl.T, device=dev)
    stream = torch.cuda.current_stream()
    for call in range(2):
        d_u = torch.full((wl.n_x * wl.T.size,), float("nan"), device=dev, dtype=torch.float64)
        F.fh_synthesize_static(wl.J, float(wl.omega[-1]), d_s, d_B, d_V, d_T, d_u,
                               stream.cuda_stream)
        stream.synchronize()
        u = d_u.cpu().numpy().reshape(wl.n_x, wl.T.size)
        assert np.all(np.isfinite(u)), call
        assert rel(u, u_ref) < TOL, call
    pr.close()


def test_static_scratch_rejects_oversize():
    import torch
    from paper_1807_02718_gb300 import build
    build.build()
    dev = torch.device("cuda", 0)
    J, n_T = 2049, 300     # J * n_T = 614700 > 524288
    d_s = torch.zeros(1, device=dev, dtype=torch.float64)
    d_B = torch.zeros(2 * J, device=dev, dtype=torch.float64)
    d_V = torch.zeros(2 * J, device=dev, dtype=torch.float64)
    d_T = torch.zeros(n_T, device=dev, dtype=torch.float64)
    d_u = torch.zeros(n_T, device=dev, dtype=torch.float64)
    with pytest.raises(F.FHError) as e:
        F.fh_synthesize_static(J, 10.0, d_s, d_B, d_V, d_T, d_u)
    assert e.value.status == F.FH_EINVAL
    # too many windows for the weights kernel's shared memory at J = 2049
    K = 2049
    d_s = torch.zeros(K, device=dev, dtype=torch.float64)
    d_B = torch.zeros(2 * K * J, device=dev, dtype=torch.float64)
    d_T = torch.zeros(10, device=dev, dtype=torch.float64)
    d_u = torch.zeros(10, device=dev, dtype=torch.float64)
    with pytest.raises(F.FHError) as e:
        F.fh_synthesize_static(J, 10.0, d_s, d_B, d_V, d_T, d_u)
    assert e.value.status == F.FH_EINVAL
