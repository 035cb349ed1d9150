"""pf_energy2d_static: the energy/mass reduction for callers that cannot
allocate device memory (a host that owns all device memory through its own
allocator, a fixed device-memory budget, or a path where cudaMalloc/cudaFree
would synchronise the device).  Its scratch is a static device array inside
libpf; the caller passes only the state and a 2-double output buffer.

Checked through the C ABI against pf_energy (the context + workspace entry
point) on two calls in a row with different states, so a stale or
uncleared static scratch would show.  This file is collected last on
purpose.
"""
import pytest
import torch

import pf_inputs as G

pytestmark = pytest.mark.gpu


def test_static_scratch_energy_matches_workspace_entry_point_twice():
    import paper_2601_06079_gb300 as pf
    from paper_2601_06079_gb300 import _lib

    shape, h, W, kappa = (300, 517), (0.9, 1.1), 1.3, 0.7
    solver = pf.Solver(shape, h=h, model="ch")
    solver.set_params(W=W, kappa=kappa, mobility=1.0, dt=1e-3)
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for seed in (11, 12):
        u = torch.from_numpy(G.ch_initial(seed, shape, amp=0.3)).cuda()
        E_ref, M_ref = solver.energy(u)
        st, msg = _lib.pf_energy2d_static(u.data_ptr(), shape[1], shape[0], h[0], h[1], W, kappa,
                                          out.data_ptr(), stream)
        assert st == _lib.PF_OK, msg
        torch.cuda.synchronize()
        E, M = out.tolist()
        assert abs(E - E_ref) <= 1e-12 * abs(E_ref)
        assert abs(M - M_ref) <= 1e-12 * abs(M_ref)


def test_static_scratch_energy_rejects_bad_sizes():
    from paper_2601_06079_gb300 import _lib

    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    u = torch.zeros(16, device="cuda")
    st, msg = _lib.pf_energy2d_static(u.data_ptr(), 1, 16, 1.0, 1.0, 1.0, 1.0, out.data_ptr(), 0)
    assert st == _lib.PF_ERR_ARG and ">= 2" in msg
    st, msg = _lib.pf_energy2d_static(u.data_ptr(), 1 << 20, 1 << 12, 1.0, 1.0, 1.0, 1.0,
                                      out.data_ptr(), 0)
    assert st == _lib.PF_ERR_ARG and "too large" in msg
