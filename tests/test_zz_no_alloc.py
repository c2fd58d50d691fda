"""The allocation-free pressure solve.

For callers that cannot allocate device memory when they need a solve (a
host whose memory manager already holds the GPU's memory, a latency-critical
loop where cudaMalloc would stall, a plugin limited to memory set aside at
load time), cahn_solve_p_noalloc keeps every intermediate in one fixed
device array.  Its result must match the context-based cahn_solve of the
same system and the oracle's exact solve of L_h p = d (Eq. 4.4, gauge
<p,1>_W = 0), on two calls in a row (the array keeps the previous call's
contents).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from oracle import cahn_oracle as O
from paper_1811_11842_gb300 import binding, inputs
from paper_1811_11842_gb300 import build as B


def test_noalloc_rejects_oversized_grid_before_any_cuda_call():
    B.build()
    lib = binding.load()
    code = lib.cahn_solve_p_noalloc(512, 512, 2.0, 1.0, 1e-10, 100, ctypes.c_void_p(16),
                                    ctypes.c_void_p(16), None, None)
    assert code == binding.CAHN_ERR_ARG
    assert "66560" in binding.load().cahn_noalloc_last_error().decode()


@pytest.mark.gpu
def test_noalloc_matches_context_solve_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    binding.load()
    cases = [inputs.config_small()[0].replace(rtol=1e-13, precond=1),
             inputs.config_small()[0].replace(nx=40, ny=22, rtol=1e-13, precond=1)]
    stream = torch.cuda.current_stream()
    for k, prm in enumerate(cases):
        geo = inputs.Protrusions(h_b=0.3, centres=(1.0,), radius=0.2, seed=3)
        state = inputs.initial_state(prm.replace(eps=max(prm.eps, 2.0 / prm.ny)), geo)
        rhs = inputs.random_field(prm, seed=20 + k)
        sim = binding.Simulation([prm], [state])
        x_ref, code, _ = sim.solve(0, binding.SYS_P, rhs)
        assert code == 0
        sim.close()
        b = torch.as_tensor(rhs, device="cuda").contiguous()
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        code, st = binding.cahn_solve_p_noalloc(prm.nx, prm.ny, prm.lx, prm.ly, prm.rtol,
                                                prm.max_iters, b.data_ptr(), x.data_ptr(),
                                                stream.cuda_stream)
        assert code == 0, st
        got, ref = x.cpu().numpy(), x_ref.cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-10
        exact = O.solve_system(prm, O.init_state(prm, *state), "p", rhs)
        assert np.linalg.norm(got - exact) / np.linalg.norm(exact) <= 1e-10
        assert st["iters"][3] > 0
