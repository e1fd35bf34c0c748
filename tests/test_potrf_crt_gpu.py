"""dd Rpotrf with residue-form (tensor-core) trailing updates (GPU).

The Cholesky of Sec. 10.5's Rpotrf benchmark in outer steps of 256 columns
whose panel and trailing updates of 512 columns or more are residue-form
Rgemm / Rsyrk calls.  Pins: an integer
Cholesky factor is recovered bit-exactly (each update is exact and the
Schur complements stay integers); on an SPD matrix of condition ~1e20 the
componentwise backward error |U^T U - A| <= c n eps (|U|^T |U|) (the
classical Cholesky bound) holds on sampled entries with the residual taken
by the oracle's exact tier, the LAPACK solve ratio (< 30) holds after
Rpotrs, and the factor meets the same bounds as the FP64-pipe Rpotrf; a
failing leading minor gives LAPACK's info and leaves every later trailing
block untouched; results are deterministic; workspace and argument errors.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import datagen
import oracle
from ddcheck import EPS_DD
from gpucase import dev, host, sample_blocks

pytestmark = pytest.mark.gpu


def potrf_crt(mp, uplo, Fh, Fl):
    n = Fh.shape[0]
    F = dev((Fh, Fl))
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = mp.workspace(mp.mp_dd_Rpotrf_crt_workspace(n))
    mp.mp_dd_Rpotrf_crt(uplo, n, F, n, info, ws, ws.numel())
    torch.cuda.synchronize()
    return F, int(info.item())


def upper_factor(uplo, fh, fl):
    if uplo == "U":
        return np.triu(fh), np.triu(fl)
    return np.tril(fh).T.copy(order="F"), np.tril(fl).T.copy(order="F")


def test_workspace_size_and_threshold(cuda_lib):
    mp = cuda_lib
    assert mp.mp_dd_Rpotrf_crt_workspace(0) == 0
    assert mp.mp_dd_Rpotrf_crt_workspace(767) == 0
    assert mp.mp_dd_Rpotrf_crt_workspace(768) >= mp.mp_dd_Rsyrk_crt_workspace(512, 256)
    assert mp.mp_dd_Rpotrf_crt_workspace(1400) >= mp.mp_dd_Rsyrk_crt_workspace(1144, 256)


@pytest.mark.parametrize("uplo", ["U", "L"])
def test_integer_factor_recovered_exactly(cuda_lib, uplo):
    n = 900                            # a 644-column panel and update on the tensor cores
    g = datagen.rng(620)
    U = np.triu(g.integers(-3, 4, (n, n))).astype(np.float64)
    np.fill_diagonal(U, g.integers(1, 5, n))
    Fm = U.T @ U
    assert np.abs(Fm).max() < 2 ** 52
    F, info = potrf_crt(cuda_lib, uplo, np.asfortranarray(Fm), np.zeros((n, n), order="F"))
    assert info == 0
    fh, fl = host(F)
    if uplo == "U":
        assert np.array_equal(np.triu(fh), U) and not np.triu(fl).any()
        assert np.array_equal(np.tril(fh, -1), np.tril(Fm, -1))    # the other triangle
    else:
        assert np.array_equal(np.tril(fh), U.T) and not np.tril(fl).any()
        assert np.array_equal(np.triu(fh, 1), np.triu(Fm, 1))


def spd_problem(seed, n):
    G, B = datagen.spd_request(seed, n)
    Fd = oracle.dd_syrk("U", "N", (1.0, 0.0), G, (0.0, 0.0),
                        (np.zeros((n, n), order="F"), np.zeros((n, n), order="F")))
    Fs = tuple(np.asfortranarray(np.triu(P) + np.triu(P, 1).T) for P in Fd)
    return G, B, Fs


def componentwise_ratio(Ut, Fs, rows, cols):
    """max |U^T U - A|_ij / (n eps (|U|^T |U|)_ij) with the residual exact."""
    n = Fs[0].shape[0]
    R = oracle.exact_gemm_entries("T", "N", n, (1.0, 0.0), Ut, Ut, (-1.0, 0.0), Fs, rows, cols)
    aU = np.abs(Ut[0])
    scale = np.einsum("ki,ki->i", aU[:, rows], aU[:, cols])
    return float((np.abs(R[0]) / (n * EPS_DD * scale)).max())


@pytest.mark.parametrize("uplo", ["U", "L"])
def test_ill_conditioned_backward_error_and_solve(cuda_lib, uplo):
    mp = cuda_lib
    n = 800
    G, B, Fs = spd_problem(621, n)
    F, info = potrf_crt(mp, uplo, *Fs)
    assert info == 0
    Ut = upper_factor(uplo, *host(F))
    rows, cols = sample_blocks(n, n, bs=32, count=8, seed=622)
    keep = rows <= cols
    rows, cols = rows[keep], cols[keep]
    assert componentwise_ratio(Ut, Fs, rows, cols) < 30
    # the FP64-pipe Rpotrf meets the same bound on the same entries
    Fp = dev(Fs)
    info_p = torch.zeros(1, dtype=torch.int64, device="cuda")
    mp.mp_dd_Rpotrf(uplo, n, Fp, n, info_p)
    assert int(info_p.item()) == 0
    assert componentwise_ratio(upper_factor(uplo, *host(Fp)), Fs, rows, cols) < 30
    # solve: the LAPACK ratio ||B - A X|| / (||A|| ||X|| eps) < 30
    X = dev(B)
    mp.mp_dd_Rpotrs(uplo, n, 4, F, n, X, n)
    xh, xl = host(X)
    rr, cc = np.meshgrid(np.arange(n), np.arange(4), indexing="ij")
    R = oracle.exact_gemm_entries("N", "N", n, (-1.0, 0.0), Fs, (xh, xl), (1.0, 0.0), B,
                                  rr.ravel(), cc.ravel())
    fn = np.abs(Fs[0]).sum(axis=0).max()
    xn = np.abs(xh).sum(axis=0).max()
    assert np.abs(R[0].reshape(n, 4)).sum(axis=0).max() / (fn * xn * EPS_DD) < 30


@pytest.mark.parametrize("uplo,fail_at", [("U", 10), ("L", 100), ("U", 600)])
def test_failing_minor_info_and_untouched_trailing_block(cuda_lib, uplo, fail_at):
    n = 1200
    Fm = np.eye(n) * 4.0
    Fm[fail_at - 1, fail_at - 1] = -5.0
    # couple the failing row to the last one: an update after the failure
    # would change the last diagonal entry
    Fm[fail_at - 1, n - 1] = Fm[n - 1, fail_at - 1] = 1.0
    F, info = potrf_crt(cuda_lib, uplo, np.asfortranarray(Fm), np.zeros((n, n), order="F"))
    assert info == fail_at
    fh, fl = host(F)
    j = (fail_at - 1) // 64 * 64        # the failing diagonal block starts here
    # every block factored before it: diag(2); no update reached later blocks
    assert np.array_equal(np.diag(fh)[:j], np.full(j, 2.0))
    after = j + 64
    assert np.array_equal(fh[after:, after:], Fm[after:, after:])
    assert not fl[after:, after:].any()


def test_deterministic(cuda_lib):
    n = 800
    _, _, Fs = spd_problem(623, n)
    a, _ = potrf_crt(cuda_lib, "L", *Fs)
    b, _ = potrf_crt(cuda_lib, "L", *Fs)
    ah, al = host(a)
    bh, bl = host(b)
    assert np.array_equal(ah, bh) and np.array_equal(al, bl)


def test_errors_and_quick_return(cuda_lib):
    mp = cuda_lib
    n = 800
    F = dev((np.eye(n), np.zeros((n, n))))
    info = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    need = mp.mp_dd_Rpotrf_crt_workspace(n)
    ws = mp.workspace(need)
    assert mp.mp_dd_Rpotrf_crt("X", n, F, n, info, ws, need, check=False) == -1
    assert mp.mp_dd_Rpotrf_crt("U", -1, F, n, info, ws, need, check=False) == -2
    assert mp.mp_dd_Rpotrf_crt("U", n, (None, None), n, info, ws, need, check=False) == -3
    assert mp.mp_dd_Rpotrf_crt("U", n, F, n - 1, info, ws, need, check=False) == -4
    assert mp.mp_dd_Rpotrf_crt("U", n, F, n, None, ws, need, check=False) == -5
    assert mp.mp_dd_Rpotrf_crt("U", n, F, n, info, None, 0, check=False) == 2003
    assert mp.mp_dd_Rpotrf_crt("U", n, F, n, info, ws, need - 1, check=False) == 2003
    # n = 0 resets info; n < 768 needs no workspace (the FP64-pipe path)
    assert mp.mp_dd_Rpotrf_crt("U", 0, F, 1, info, None, 0, check=False) == 0
    assert int(info.item()) == 0
    S = dev((np.eye(300) * 9.0, np.zeros((300, 300))))
    assert mp.mp_dd_Rpotrf_crt("L", 300, S, 300, info, None, 0, check=False) == 0
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert np.array_equal(np.diag(host(S)[0]), np.full(300, 3.0))
