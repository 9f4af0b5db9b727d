"""Every device call of a handle checks that the handle's device is the
current one (a handle's buffers, stream and graphs live on the device that
was current at create).  With one GPU the mismatch is made with the test
hook that overwrites the ordinal recorded in the handle: each call must then
return ERR_ARG naming both ordinals, without touching the device, and the
handle must work again once the true ordinal is back."""
import numpy as np
import pytest

import synth
from conftest import has_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]


def test_calls_refused_on_another_device():
    import torch
    import paper_2109_00485_gb300 as pkg
    pkg.load()
    A = synth.tile_matrix(700, 30, seed=41, fp32=True)
    h = pkg.from_csr(A, k=8, nev=2)
    X = torch.from_numpy(synth.normal_block(A.n, 8, seed=3, fp32=True)).cuda()
    Y_ref = h.spmm_sym(X)
    HS = Y_ref
    theta = torch.zeros(8, dtype=torch.float64, device="cuda")
    C = torch.zeros((8, 4), dtype=torch.float64, device="cuda")
    th = torch.zeros(4, dtype=torch.float64, device="cuda")
    true_dev = torch.cuda.current_device()
    h.lobpcg_test_set_device_ordinal(true_dev + 7)
    calls = {
        "spmm_sym": lambda: h.spmm_sym(X),
        "precond_apply": lambda: h.precond_apply(X, theta, mode="diag"),
        "rayleigh_ritz": lambda: h.rayleigh_ritz(X, HS, 4),
        "rayleigh_ritz_noalloc": lambda: h.rayleigh_ritz_noalloc(X, HS, 4, C, th),
        "sync": lambda: h.sync(),
    }
    for name, call in calls.items():
        with pytest.raises(pkg.LobpcgError) as e:
            call()
        assert e.value.status == 1, name
        assert f"device {true_dev + 7}" in str(e.value) and f"device {true_dev}" in str(e.value), (name, str(e.value))
    with pytest.raises(pkg.LobpcgError) as e:
        h.solve(synth.initial_guess(A, 8, seed=5, fp32=True))
    assert e.value.status == 1
    h.lobpcg_test_set_device_ordinal(true_dev)
    Y = h.spmm_sym(X)
    C2, th2 = h.rayleigh_ritz(X, HS, 4)
    h.rayleigh_ritz_noalloc(X, HS, 4, C, th)
    assert torch.allclose(th, th2, rtol=1e-10, atol=0)
    torch.cuda.synchronize()
    assert np.allclose(Y.cpu().numpy(), Y_ref.cpu().numpy(), rtol=1e-5, atol=1e-5)
    h.destroy()
