"""lobpcg_rayleigh_ritz_noalloc (static scratch, no allocation) against
lobpcg_rayleigh_ritz on the same inputs, two calls in a row with different
subspaces so that the second call starts from the first one's leftovers in
the shared scratch array; and its size limit."""
import numpy as np
import pytest

import synth
from conftest import has_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]


def _pkg():
    import paper_2109_00485_gb300 as pkg
    pkg.load()
    return pkg


def _same_pairs(C1, t1, C2, t2):
    assert np.allclose(t1, t2, rtol=1e-10, atol=1e-12 * np.abs(t2).max())
    # eigenvectors up to sign
    for j in range(C1.shape[1]):
        s = np.sign(C1[:, j] @ C2[:, j]) or 1.0
        assert np.allclose(C1[:, j], s * C2[:, j], rtol=0, atol=1e-7 * np.abs(C2[:, j]).max())


def test_noalloc_matches_allocating_entry_twice_in_a_row():
    import torch
    pkg = _pkg()
    A = synth.tile_matrix(3000, 50, seed=31, fp32=True)
    h = pkg.from_csr(A, k=8, nev=1)
    for call, (m, k, seed) in enumerate(((24, 8, 1), (32, 10, 2))):
        S = torch.from_numpy(synth.normal_block(A.n, m, seed=seed, fp32=True)).cuda()
        HS = h.spmm_sym(S)
        C_ref, th_ref = h.rayleigh_ritz(S, HS, k)
        C = torch.full((m, k), np.nan, dtype=torch.float64, device="cuda")
        th = torch.full((k,), np.nan, dtype=torch.float64, device="cuda")
        h.rayleigh_ritz_noalloc(S, HS, k, C, th)
        _same_pairs(C.cpu().numpy(), th.cpu().numpy(), C_ref.cpu().numpy(), th_ref.cpu().numpy())
    h.destroy()


def test_noalloc_rejects_oversize():
    import torch
    pkg = _pkg()
    A = synth.tile_matrix(500, 20, seed=32, fp32=True)
    h = pkg.from_csr(A, k=4, nev=1)
    m, k = 97, 4
    S = torch.zeros((A.n, m), dtype=torch.float32, device="cuda")
    C = torch.zeros((m, k), dtype=torch.float64, device="cuda")
    th = torch.zeros((k,), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.LobpcgError) as e:
        h.rayleigh_ritz_noalloc(S, S, k, C, th)
    assert e.value.status == 1 and "m <= 96" in str(e.value)
    h.destroy()
