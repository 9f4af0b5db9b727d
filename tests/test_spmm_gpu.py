"""Parity of the CUDA symmetric SpMM (through the C ABI) with the CPU oracle.

Tolerance (float32 products and accumulation; the oracle is float64 on the
same inputs): componentwise |y - y_oracle| <= 1e-5 (|H| |X|)_ij and per
column ||y - y_oracle|| / ||y_oracle|| <= 1e-5.  The float64-vector product
(compensated float32 for even k <= 32, float64 arithmetic otherwise) must
agree to 1e-12 (|H| |X|)_ij."""
import numpy as np
import pytest

import oracle
import synth
from conftest import has_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]


def _pkg():
    import paper_2109_00485_gb300 as pkg
    pkg.load()
    return pkg


def abs_csr(A):
    return synth.CSR(n=A.n, row_ptr=A.row_ptr, col=A.col, val=np.abs(A.val))


def check(A, X, Y, rtol=1e-5):
    Xd = np.asarray(X, dtype=np.float64)
    Yo = oracle.spmm_tri(A, Xd)
    scale = oracle.spmm_tri(abs_csr(A), np.abs(Xd))
    Yg = np.asarray(Y, dtype=np.float64)
    err = np.abs(Yg - Yo)
    worst = np.max(err / (scale + 1e-300)) if err.size else 0.0
    assert np.all(err <= rtol * scale + 1e-30), f"componentwise scaled error {worst:.3e}"
    cn = np.linalg.norm(Yo, axis=0)
    ce = np.linalg.norm(Yg - Yo, axis=0)
    ok = cn > 0
    assert np.all(ce[ok] <= rtol * cn[ok]), f"column errors {ce[ok] / cn[ok]}"
    assert np.all(ce[~ok] == 0)


def run(A, k, seed=7, fp32_vals=None, **kw):
    import torch
    pkg = _pkg()
    X = synth.normal_block(A.n, k, seed=seed, fp32=True)
    h = pkg.from_csr(A, k=min(k, 32), nev=1, **kw)
    Y = h.spmm_sym(torch.from_numpy(X).cuda())
    h.sync()
    out = Y.cpu().numpy()
    h.destroy()
    return X, out


def test_small_workload_n20k_fp64_values():
    p = synth.WORKLOADS["small_n20k"]
    A = synth.tile_matrix(p["n"], p["nnz_per_row"], seed=p["seed"], fp32=False)
    X, Y = run(A, p["k"])
    # the GPU stores float32 values: compare against the oracle on the same rounding
    A32 = synth.CSR(n=A.n, row_ptr=A.row_ptr, col=A.col, val=A.val.astype(np.float32))
    check(A32, X, Y)
    check(A, X, Y, rtol=2e-5)


@pytest.mark.parametrize("k", [1, 3, 4, 8, 12, 16, 20, 32])
def test_ragged_n_all_k(k):
    A = synth.tile_matrix(2003, 120, seed=5, fp32=True)
    X, Y = run(A, k)
    check(A, X, Y)


@pytest.mark.parametrize("n", [1, 2, 15, 16, 17, 33, 300])
def test_tiny_sizes(n):
    A = synth.tile_matrix(n, 40, seed=n, fp32=True)
    for k in (4, 16):
        X, Y = run(A, k)
        check(A, X, Y)


def _random_lower(n, density, seed, empty=()):
    rng = np.random.default_rng(seed)
    a = np.zeros((n, n))
    m = rng.random((n, n)) < density
    a[m] = rng.standard_normal(m.sum())
    a = np.tril(a)
    np.fill_diagonal(a, rng.uniform(0, 10, n))
    for i in empty:
        a[i, :] = 0
        a[:, i] = 0
    rows, cols = np.nonzero(a)
    keep = rows >= cols
    rows, cols = rows[keep], cols[keep]
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    return synth.CSR(n=n, row_ptr=np.cumsum(rp), col=cols.astype(np.int32),
                     val=a[rows, cols].astype(np.float32))


@pytest.mark.parametrize("k", [4, 8, 16, 5])
def test_partial_chunks_and_empty_rows(k):
    A = _random_lower(700, 0.03, seed=3, empty=(0, 1, 2, 350, 699))
    X, Y = run(A, k)
    check(A, X, Y)
    assert np.all(Y[[0, 1, 2, 350, 699]] == 0)


def test_diagonal_only():
    n = 1000
    d = np.linspace(-5, 5, n).astype(np.float32)
    A = synth.CSR(n=n, row_ptr=np.arange(n + 1, dtype=np.int64), col=np.arange(n, dtype=np.int32), val=d)
    X, Y = run(A, 8)
    exact = d[:, None].astype(np.float64) * X
    # one product per output: the split product's error bound (3 * 2^-20
    # relative) plus one float32 rounding, inside the 1e-5 SpMM tolerance
    assert np.all(np.abs(Y - exact) <= 4e-6 * np.abs(exact))


def test_long_row_over_4096_entries():
    """An arrow matrix: the last row couples to every column (5000 > 4096 entries)."""
    n = 5000
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:n] = np.arange(1, n)
    rp[n] = (n - 1) + n
    cols = np.concatenate([np.arange(n - 1), np.arange(n)]).astype(np.int32)
    rng = np.random.default_rng(1)
    vals = np.concatenate([rng.uniform(1, 2, n - 1), rng.standard_normal(n)]).astype(np.float32)
    A = synth.CSR(n=n, row_ptr=rp, col=cols, val=vals)
    for k in (8, 16, 7):
        X, Y = run(A, k)
        check(A, X, Y)


def test_device_csr_input_and_repeat():
    import torch
    pkg = _pkg()
    A = synth.tile_matrix(4099, 90, seed=9, fp32=True)
    h = pkg.lobpcg_create(A.n, torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col).cuda(),
                          torch.from_numpy(A.val).cuda(), k=16, nev=4)
    X = synth.normal_block(A.n, 16, seed=2, fp32=True)
    Xd = torch.from_numpy(X).cuda()
    Y1 = h.spmm_sym(Xd).cpu().numpy()
    Y2 = h.spmm_sym(Xd).cpu().numpy()
    h.sync()
    check(A, X, Y1)
    check(A, X, Y2)
    info = h.info()
    assert info["nnz"] == A.nnz and info["row_blocks"] == (A.n + 15) // 16
    assert info["padded_nnz"] >= A.nnz and info["full_chunks"] > 0
    assert abs(info["gershgorin"] - oracle.gershgorin(A)) <= 1e-9 * info["gershgorin"]
    h.destroy()


def test_unaligned_vectors_take_simple_path():
    import torch
    pkg = _pkg()
    A = synth.tile_matrix(1500, 60, seed=4, fp32=True)
    k = 8
    X = synth.normal_block(A.n, k, seed=3, fp32=True)
    h = pkg.from_csr(A, k=k, nev=1)
    bx = torch.zeros(A.n * k + 1, device="cuda")
    by = torch.zeros(A.n * k + 1, device="cuda")
    Xv = bx[1:].view(A.n, k)
    Yv = by[1:].view(A.n, k)
    Xv.copy_(torch.from_numpy(X))
    h.spmm_sym(Xv, Yv)
    h.sync()
    check(A, X, Yv.cpu().numpy())
    h.destroy()


@pytest.mark.parametrize("k", [5, 8, 16, 20, 32])
def test_fp64_vectors(k):
    import torch
    pkg = _pkg()
    A = synth.tile_matrix(3001, 80, seed=6, fp32=True)
    X = synth.normal_block(A.n, k, seed=8)
    h = pkg.from_csr(A, k=k, nev=1)
    Y = h.spmm_sym_f64(torch.from_numpy(X).cuda()).cpu().numpy()
    h.sync()
    Yo = oracle.spmm_tri(A, X)
    scale = oracle.spmm_tri(abs_csr(A), np.abs(X))
    assert np.all(np.abs(Y - Yo) <= 1e-12 * scale)
    h.destroy()


def test_invalid_structure_rejected():
    pkg = _pkg()
    A = synth.tile_matrix(200, 30, seed=2, fp32=True)
    bad = synth.CSR(n=A.n, row_ptr=A.row_ptr.copy(), col=A.col.copy(), val=A.val.copy())
    r = 100
    a, b = bad.row_ptr[r], bad.row_ptr[r + 1]
    bad.col[a], bad.col[a + 1] = bad.col[a + 1], bad.col[a]       # unsorted row
    with pytest.raises(pkg.LobpcgError) as ei:
        pkg.from_csr(bad, k=8, nev=1)
    assert ei.value.status == 8 and "row 100" in str(ei.value)
    up = synth.CSR(n=A.n, row_ptr=A.row_ptr.copy(), col=A.col.copy(), val=A.val.copy())
    up.col[up.row_ptr[51] - 1] = 120                               # column > row (upper entry)
    with pytest.raises(pkg.LobpcgError) as ei:
        pkg.from_csr(up, k=8, nev=1)
    assert ei.value.status == 8
    rp = A.row_ptr.copy()
    rp[-1] += 5                                                     # row_ptr[n] != nnz
    with pytest.raises(pkg.LobpcgError):
        pkg.lobpcg_create(A.n, rp, A.col, A.val, k=8, nev=1)


@pytest.mark.slow
def test_full_size_n2m_sampled_rows():
    """The bench workload (n = 2M, ~400 stored entries per row, k = 16) in the
    bench's launch configuration; sampled rows against the oracle computed
    one by one, and the symmetry identity over the whole product."""
    import torch
    pkg = _pkg()
    p = synth.WORKLOADS["full_n2m"]
    A = synth.tile_matrix(p["n"], p["nnz_per_row"], seed=p["seed"], fp32=True)
    k = p["k"]
    X1 = synth.normal_block(A.n, k, seed=31, fp32=True)
    X2 = synth.normal_block(A.n, k, seed=32, fp32=True)
    h = pkg.from_csr(A, k=k, nev=p["nev"])
    Y1 = h.spmm_sym(torch.from_numpy(X1).cuda())
    Y2 = h.spmm_sym(torch.from_numpy(X2).cuda())
    h.sync()
    rows = np.unique(np.concatenate([[0, 1, 15, 16, A.n - 1, A.n - 16],
                                     synth.u64(58, 77, 1) % np.uint64(A.n)]).astype(np.int64))
    Yo = oracle.spmm_rows(A, X1.astype(np.float64), rows)
    scale = oracle.spmm_rows(abs_csr(A), np.abs(X1).astype(np.float64), rows)
    Yg = Y1.cpu().numpy()[rows].astype(np.float64)
    assert np.all(np.abs(Yg - Yo) <= 1e-5 * scale)
    # X2^T (H X1) == (H X2)^T X1, each side accumulated in float64 on the GPU
    a = (Y1.double().T @ torch.from_numpy(X2).cuda().double()).cpu().numpy()
    b = (torch.from_numpy(X1).cuda().double().T @ Y2.double()).cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-5 * np.max(np.abs(a))
    h.destroy()


def _mixed_tiles(n, seed):
    """Lower triangle with complete 16x16 tiles, complete diagonal tiles,
    partial tiles and a partial last row block (n not a multiple of 16)."""
    A = synth.tile_matrix(n, 60, seed=seed, fp32=True)
    rng = np.random.default_rng(seed)
    keep = rng.random(A.nnz) < 0.97                 # punch holes into some tiles
    rows = np.repeat(np.arange(n), np.diff(A.row_ptr))
    keep |= rows == A.col                           # keep the diagonal
    # keep every tile of the first 40 row blocks complete
    keep |= rows < 640
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows[keep] + 1, 1)
    return synth.CSR(n=n, row_ptr=np.cumsum(rp), col=A.col[keep], val=A.val[keep])


@pytest.mark.parametrize("k", [8, 16, 20, 32, 7, 12])
def test_value_only_tiles_match_oracle(k):
    """tile_format 1 (complete tiles and complete diagonal triangles keep
    value words only): tiled kernel (k % 4 == 0) and simple kernel (other k)
    against the oracle, and bit-for-bit equal to tile_format 0 on the
    simple kernel's float64 path."""
    import torch
    A = _mixed_tiles(3001, seed=31)
    X, Y = run(A, k, tile_format=1)
    check(A, X, Y)
    pkg = _pkg()
    h = pkg.from_csr(A, k=min(k, 32), nev=1, tile_format=1)
    info = h.info()
    assert info["tile_format"] == 1 and info["full_chunks"] > 0
    Xd = torch.from_numpy(X.astype(np.float64)).cuda()
    Y64 = h.spmm_sym_f64(Xd).cpu().numpy()
    h.destroy()
    h0 = pkg.from_csr(A, k=min(k, 32), nev=1)
    Y64b = h0.spmm_sym_f64(Xd).cpu().numpy()
    info0 = h0.info()
    h0.destroy()
    Yo = oracle.spmm_tri(A, X.astype(np.float64))
    scale = oracle.spmm_tri(abs_csr(A), np.abs(X.astype(np.float64)))
    assert np.all(np.abs(Y64 - Yo) <= 1e-12 * scale + 1e-300)
    assert np.all(np.abs(Y64b - Yo) <= 1e-12 * scale + 1e-300)
    # value-only storage: every complete tile saves its 256 index words
    assert info["stream_bytes"] < info0["stream_bytes"] - 4 * 256 * info["full_chunks"] + 1


def test_value_only_full_workload_rows_sampled():
    """tile_format 1 on a 400-per-row matrix (every off-diagonal tile complete),
    n = 200,016, k = 16: all rows against the oracle."""
    A = synth.tile_matrix(200016, 400, seed=2, fp32=True)
    X, Y = run(A, 16, tile_format=1)
    check(A, X, Y)
